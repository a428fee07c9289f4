"""Lagrange-parameter sweep (the selection procedure of Secs. 3.1.3 and 5).

The paper runs the joint inversion with fixed (lambda1, lambda2) for a short list of
increasing pairs and keeps the smallest pair whose models are correlated (seen in
the density-susceptibility cross-plot) and fit both data sets.  Here every pair is
one solver; all of them advance together in one batched CUDA graph
(gj_rrcg_batch_*).  Each pair gets its own operators because an operator's
workspace cannot be shared by concurrent solvers.  The correlation of the final
models is reported as a Pearson coefficient (gj_pearson, on the device).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np
import torch

from .api import Batch, Solver, bttb_setup, solver_params


def pearson(a, b, stream=None) -> float:
    """Pearson coefficient of two models (gj_pearson on the device; numpy arrays are
    copied to the device first).  Returns a float."""
    import ctypes as ct

    from . import _lib
    from .api import _ptr, _stream

    ta = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    tb = b if isinstance(b, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(b, dtype=np.float64))
    ta = ta.cuda().contiguous()
    tb = tb.to(device=ta.device, dtype=ta.dtype).contiguous()
    if ta.dtype not in (torch.float32, torch.float64) or ta.numel() != tb.numel():
        raise ValueError("pearson: two float32 or float64 vectors of one length")
    prec = _lib.GJ_FP64 if ta.dtype == torch.float64 else _lib.GJ_FP32_MIXED
    r = torch.empty(1, dtype=torch.float64, device=ta.device)
    _lib.check(_lib.load().gj_pearson(ta.numel(), prec, _ptr(ta), _ptr(tb), _ptr(r), _stream(stream)))
    return float(r.item())


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
        r = pearson(m[0], m[1])
        m1 = m[0].double().cpu().numpy()
        m2 = m[1].double().cpu().numpy()
        runs.append({"lambda": [float(lam[0]), float(lam[1])], "iterations": rep["iterations"],
                     "converged": rep["converged"], "phi": rep["phi"], "S_G": rep["S_G"],
                     "pearson": r, "models": (m1, m2)})
        s.close()
        for o in ops:
            o.close()
    selected = None
    for i, r in enumerate(runs):
        if r["converged"] and r["pearson"] >= corr_threshold:
            selected = i
            break
    return {"runs": runs, "selected": selected}
