"""Lagrange-parameter sweep (the selection procedure of Secs. 3.1.3 and 5).

The paper runs the joint inversion with fixed (lambda1, lambda2) for a short list of
increasing pairs and keeps the smallest pair whose models are correlated (seen in
the density-susceptibility cross-plot) and fit both data sets.  Here every pair is
one solver; all of them advance together in one batched CUDA graph
(gj_rrcg_batch_*).  Each pair gets its own operators because an operator's
workspace cannot be shared by concurrent solvers.  The correlation of the final
models is reported as a Pearson coefficient, computed on the host.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np
import torch

from .api import Batch, Solver, bttb_setup, solver_params


def pearson(a: np.ndarray, b: np.ndarray) -> float:
    a = np.asarray(a, dtype=np.float64) - np.mean(a)
    b = np.asarray(b, dtype=np.float64) - np.mean(b)
    den = np.sqrt((a @ a) * (b @ b))
    return float(a @ b / den) if den > 0 else 0.0


def lambda_sweep(grid, mag, dobs, sigma, w_depth, lambdas: Sequence[Tuple[float, float]], precision: str = "fp32",
                 npad=(0, 0), corr_threshold: float = 0.9, chunk: int = 10, **params) -> Dict:
    """Runs one joint solve per (lambda1, lambda2) in ``lambdas`` (ordered from small to
    large) and returns {"runs": [...], "selected": index or None}.  ``dobs``, ``sigma``
    and ``w_depth`` are pairs of device tensors; ``params`` go to solver_params."""
    kmax = params.get("kmax", 50)
    runs, solvers, keep = [], [], []
    for lam in lambdas:
        ops = [bttb_setup(grid, "gravity", None, precision, npad), bttb_setup(grid, "magnetic", mag, precision, npad)]
        m = [torch.zeros(ops[0].n, dtype=ops[0].dtype, device=dobs[0].device) for _ in range(2)]
        P = solver_params(lam=tuple(float(x) for x in lam), **params)
        solvers.append(Solver(ops, P, dobs, sigma, w_depth, m))
        keep.append((ops, m))
    batch = Batch(solvers)
    done_iters = 0
    while done_iters < kmax and not batch.all_done():
        step = min(chunk, kmax - done_iters)
        batch.step(step)
        done_iters += step
    batch.close()
    for lam, s, (ops, m) in zip(lambdas, solvers, keep):
        rep = s.report()
        m1 = m[0].double().cpu().numpy()
        m2 = m[1].double().cpu().numpy()
        runs.append({"lambda": [float(lam[0]), float(lam[1])], "iterations": rep["iterations"],
                     "converged": rep["converged"], "phi": rep["phi"], "S_G": rep["S_G"],
                     "pearson": pearson(m1, m2), "models": (m1, m2)})
        s.close()
        for o in ops:
            o.close()
    selected = None
    for i, r in enumerate(runs):
        if r["converged"] and r["pearson"] >= corr_threshold:
            selected = i
            break
    return {"runs": runs, "selected": selected}
