"""Regularised reweighted conjugate gradient joint solve (oracle; FP64).

Follows Sec. 2.4 (Eq. RRCG:1-8), the bound projection of Sec. 2.5, the chi^2
termination of Sec. 2.6 (Eq. chi2) and the alpha schedule of Sec. 2.8
(Eq. regpara), one step at a time, with dense (or any exact) matvecs passed in.

Readings where the paper is silent or ambiguous (each listed in the design notes):
* RRCG:4 regulariser anchor: the printed difference uses the previous weighted
  model, while the first variation (Eq. FirstVariation) has m~ - m~_apr.  The
  default anchor is m~_apr = W_k m_apr, which makes the lambda = 0, p = 2, fixed
  alpha case exact linear CG; anchor="previous" keeps the printed form.
* Scalars: the overbars are concatenations, so one beta_k and one s_k serve both
  fields ("joint"); for lambda = 0 the paper runs each field stand-alone
  ("per_field"), with its own beta and s.
* RRCG:6 denominator: sum_i ||A~_i p_i||^2 + alpha_i ||p_i||^2 + lambda_i ||p_i||^2,
  as printed.
* W_k is recomputed from m_k at every iteration; p_{k-1} and ||l_{k-1}||^2 carry
  over (no restart); p_0 = l_0.
* Order: at iteration k the residual of m_k gives Phi_k (Eq. chi2); a field whose
  Phi_k <= s + sqrt(2 s) is marked satisfied for good and its alpha is frozen;
  otherwise alpha_k = max(q alpha_{k-1}, alpha_min) for k >= 1 (alpha_0 = alpha1).
  The solve stops before updating when both fields are satisfied (if stopping is
  enabled) or when k = K_max.  The model update is clipped to [lo, hi] after RRCG:8.
* Gramian space: "original" uses RRCG:2-3 on the unweighted models (the paper's
  default); "weighted" uses Eq. steepestascenta/b on m~ = W m.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np

from .gramian import ascent_directions, gramian
from .weights import lp_weight


@dataclass
class RRCGParams:
    p: Sequence[int] = (1, 1)
    eps2: float = 1e-9
    alpha1: Sequence[float] = (2.0e4, 2.0e4)
    q: Sequence[float] = (0.95, 0.95)
    alpha_min: Sequence[float] = (0.0, 0.0)
    lam: Sequence[float] = (0.0, 0.0)
    lo: Sequence[float] = (0.0, 0.0)
    hi: Sequence[float] = (1.0, 0.1)
    kmax: int = 50
    stop_on_chi2: bool = True
    scalars: str = "auto"          # "joint", "per_field" or "auto" (per_field iff lambda == 0)
    anchor: str = "apriori"        # or "previous"
    gramian_space: str = "original"  # or "weighted"


@dataclass
class RRCGResult:
    m: List[np.ndarray]
    iterations: int
    converged: bool
    satisfied: List[bool]
    history: List[dict] = field(default_factory=list)


def rrcg_joint(fwd: Sequence[Callable], adj: Sequence[Callable], d_obs, sigma, m0,
               w_static, params: RRCGParams, m_apr=None) -> RRCGResult:
    """Joint RRCG for two fields.

    fwd[i](x) = A^(i) x and adj[i](y) = A^(i)T y; d_obs[i], sigma[i] data and their
    standard deviations (W_d = 1 / sigma); m0[i] the starting models; w_static[i]
    the per-cell product W_depth W_hard (a vector of length n).
    """
    P = params
    nf = 2
    wd = [1.0 / np.asarray(sigma[i], dtype=np.float64) for i in range(nf)]
    dob = [np.asarray(d_obs[i], dtype=np.float64) for i in range(nf)]
    m = [np.array(m0[i], dtype=np.float64) for i in range(nf)]
    mapr = [np.zeros_like(m[i]) if m_apr is None or m_apr[i] is None
            else np.asarray(m_apr[i], dtype=np.float64) for i in range(nf)]
    ws = [np.asarray(w_static[i], dtype=np.float64) for i in range(nf)]
    per_field = (P.scalars == "per_field") or (P.scalars == "auto" and all(l == 0 for l in P.lam))
    s_count = [dob[i].size for i in range(nf)]
    chi2_target = [s_count[i] + np.sqrt(2.0 * s_count[i]) for i in range(nf)]

    alpha = [float(a) for a in P.alpha1]
    sat = [False, False]
    p_prev = None
    ll_prev = None
    mt_prev = None
    hist = []
    k = 0
    while True:
        # RRCG:1 on the current model (A~ m~ = W_d A m)
        rt = [wd[i] * (fwd[i](m[i]) - dob[i]) for i in range(nf)]
        phi = [float(rt[i] @ rt[i]) for i in range(nf)]
        for i in range(nf):
            if phi[i] <= chi2_target[i]:
                sat[i] = True
        if k > 0:
            for i in range(nf):
                if not sat[i]:
                    alpha[i] = max(P.q[i] * alpha[i], P.alpha_min[i])
        # W_k from m_k (Eq. W, Eq. WL)
        W = [ws[i] * lp_weight(m[i], mapr[i], P.eps2, P.p[i]) for i in range(nf)]
        mt = [W[i] * m[i] for i in range(nf)]
        # S_G of the original models, and of the models in the Gramian's space
        # (Appendix A: the weighted-space Gramian of W m)
        sg_space = gramian(m[0], m[1]) if P.gramian_space == "original" else gramian(mt[0], mt[1])
        rec = {"k": k, "phi": phi, "alpha": list(alpha), "S_G": gramian(m[0], m[1]), "S_G_space": sg_space,
               "satisfied": list(sat)}
        hist.append(rec)
        if (P.stop_on_chi2 and all(sat)) or k >= P.kmax:
            break

        if P.anchor == "apriori":
            anchor = [W[i] * mapr[i] for i in range(nf)]
        else:
            anchor = [mt_prev[i] if mt_prev is not None else W[i] * mapr[i] for i in range(nf)]

        # RRCG:2-3 (or Eq. steepestascenta/b in the weighted space)
        if P.gramian_space == "original":
            lG = ascent_directions(m[0], m[1])
        else:
            lG = ascent_directions(mt[0], mt[1])

        # RRCG:4: A~^T r~ = W^-1 A^T (W_d r~)
        l = [adj[i](wd[i] * rt[i]) / W[i] + alpha[i] * (mt[i] - anchor[i]) + P.lam[i] * lG[i]
             for i in range(nf)]
        ll = [float(l[i] @ l[i]) for i in range(nf)]

        # RRCG:5
        if p_prev is None:
            p = [l[i].copy() for i in range(nf)]
            beta = [0.0, 0.0]
        else:
            if per_field:
                beta = [ll[i] / ll_prev[i] if ll_prev[i] > 0 else 0.0 for i in range(nf)]
            else:
                den = ll_prev[0] + ll_prev[1]
                b = (ll[0] + ll[1]) / den if den > 0 else 0.0
                beta = [b, b]
            p = [l[i] + beta[i] * p_prev[i] for i in range(nf)]

        # RRCG:6: A~ p = W_d A (W^-1 p)
        qv = [wd[i] * fwd[i](p[i] / W[i]) for i in range(nf)]
        num = [float(p[i] @ l[i]) for i in range(nf)]
        den = [float(qv[i] @ qv[i]) + (alpha[i] + P.lam[i]) * float(p[i] @ p[i]) for i in range(nf)]
        if per_field:
            s = [num[i] / den[i] if den[i] > 0 else 0.0 for i in range(nf)]
        else:
            tot = den[0] + den[1]
            sj = (num[0] + num[1]) / tot if tot > 0 else 0.0
            s = [sj, sj]

        # RRCG:7-8 and the bound projection of Sec. 2.5
        for i in range(nf):
            m[i] = np.clip(m[i] - s[i] * p[i] / W[i], P.lo[i], P.hi[i])
        rec.update({"beta": beta, "s": s, "ll": ll, "pl": num, "den": den})
        p_prev, ll_prev, mt_prev = p, ll, mt
        k += 1

    return RRCGResult(m=m, iterations=k, converged=all(sat), satisfied=list(sat), history=hist)

