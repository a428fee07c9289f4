"""Padded-size autotuner for the BCCB embedding.

Any padded size N >= s + n - 1 gives the same product (Sec. 2.7.1), so the choice
is purely a speed question: the FFT radix plan follows from N's factors, and a
512 x 512 embedding (for up to 256 prisms and stations per direction, FP32)
selects the specialised warp-FFT kernels.  ``tune`` times one forward and one
adjoint product of both fields for each candidate size with CUDA events, keeps
the fastest, and caches the choice in a JSON file keyed by the grid sizes and
precision.
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Optional, Tuple

import torch

from .api import bttb_setup


def smooth_sizes(minimum: int, count: int = 3, primes=(2, 3, 5, 7)) -> List[int]:
    """The first ``count`` integers >= minimum whose prime factors are all in ``primes``."""
    out = []
    n = max(1, minimum)
    while len(out) < count and n <= 2048:
        m = n
        for p in primes:
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
        n += 1
    return out


def candidates(grid, precision: str) -> List[Tuple[int, int]]:
    ys = smooth_sizes(grid.sy + grid.ny - 1)
    xs = smooth_sizes(grid.sx + grid.nx - 1)
    cands = list(zip(ys, xs))
    if precision == "fp32" and max(grid.sx, grid.sy, grid.nx, grid.ny) <= 256 and (512, 512) not in cands:
        cands.append((512, 512))
    return cands


def _key(grid, precision) -> str:
    return (f"s{grid.sx}x{grid.sy}-n{grid.nx}x{grid.ny}x{grid.nz}-off{getattr(grid, 'off_x', 0)},"
            f"{getattr(grid, 'off_y', 0)}-{precision}")


def _time_pair(grid, mag, precision, npad, reps) -> float:
    ops = [bttb_setup(grid, "gravity", None, precision, npad), bttb_setup(grid, "magnetic", mag, precision, npad)]
    dt = ops[0].dtype
    m = torch.rand(ops[0].n, dtype=dt, device="cuda")
    r = torch.randn(ops[0].s, dtype=dt, device="cuda")
    d = torch.empty(ops[0].s, dtype=dt, device="cuda")
    g = torch.empty(ops[0].n, dtype=dt, device="cuda")
    for op in ops:  # warm-up
        op.forward(m, d)
        op.adjoint(r, g)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        for op in ops:
            op.forward(m, d)
            op.adjoint(r, g)
    e1.record()
    e1.synchronize()
    for op in ops:
        op.close()
    return e0.elapsed_time(e1) / reps


def tune(grid, mag, precision: str = "fp32", cache: Optional[str] = None, reps: int = 5) -> Tuple[int, int]:
    """Returns (Npad_y, Npad_x) for this grid and precision (cached in ``cache``)."""
    table: Dict[str, dict] = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    key = _key(grid, precision)
    if key in table:
        return tuple(table[key]["npad"])
    timings = {}
    for cand in candidates(grid, precision):
        timings[f"{cand[0]}x{cand[1]}"] = _time_pair(grid, mag, precision, cand, reps)
    best = min(timings, key=timings.get)
    npad = tuple(int(v) for v in best.split("x"))
    table[key] = {"npad": list(npad), "ms_fwd_adj_both_fields": timings}
    if cache:
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return npad
