"""Autotuner of the BCCB embedding: padded size, radix plan and launch shapes.

Any padded size N >= s + n - 1 gives the same product (Sec. 2.7.1), so the choice
is purely a speed question: a 512 x 512 embedding (for up to 256 prisms and
stations per direction, FP32), or 256 x 512 (at most 128 of them along y), selects
the specialised warp-FFT kernels; other
sizes run the general kernels, whose radix plan and tiles (line pairs per CTA of
the row passes, columns per CTA of the column passes, layers per CTA of the
spectrum multiply; gj_op_tune) are searched too.  ``tune_full`` times one forward
and one adjoint product of both fields with CUDA events for each candidate size,
then refines the best general size one knob at a time, keeps the fastest overall,
and caches the choice in a JSON file keyed by the grid sizes and precision.
``tune`` returns only the padded size.
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
    if precision == "fp32" and max(grid.sx, grid.nx) <= 256:
        # the specialised kernels: N_x = 512, and N_y = 512 or, for at most 128
        # stations and prisms per column, 256
        if max(grid.sy, grid.ny) <= 256 and (512, 512) not in cands:
            cands.append((512, 512))
        if max(grid.sy, grid.ny) <= 128 and (256, 512) not in cands:
            cands.append((256, 512))
    return cands


def _key(grid, precision) -> str:
    return (f"s{grid.sx}x{grid.sy}-n{grid.nx}x{grid.ny}x{grid.nz}-off{getattr(grid, 'off_x', 0)},"
            f"{getattr(grid, 'off_y', 0)}-{precision}")


def _time_ops(ops, reps) -> float:
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
    return e0.elapsed_time(e1) / reps


def _setup(grid, mag, precision, npad):
    return [bttb_setup(grid, "gravity", None, precision, npad), bttb_setup(grid, "magnetic", mag, precision, npad)]


# knob values searched for the general kernels (invalid shapes are skipped)
KNOBS = {"P_row": (1, 2, 4, 8, 16), "C_col": (1, 2, 4, 8, 16), "L_grp": (1, 2, 4, 8), "radix_order": (0, 1, 2)}


def _refine(ops, reps, base_ms):
    """One pass of coordinate search over KNOBS on the general kernels; returns the
    settings that differ from the library's defaults and the tuned time."""
    from ._lib import GJError

    default = ops[0].tiles()
    cur_set = dict(default)
    cur = base_ms
    for knob, values in KNOBS.items():
        for v in values:
            if v == cur_set[knob]:
                continue
            try:
                for op in ops:
                    op.tune(**{knob: v})
            except GJError:
                continue
            t = _time_ops(ops, reps)
            if t < cur * 0.98:
                cur, cur_set[knob] = t, v
        for op in ops:  # leave the knob at its best value for the next one
            op.tune(**{knob: cur_set[knob]})
    return {k: v for k, v in cur_set.items() if v != default[k]}, cur


def tune_full(grid, mag, precision: str = "fp32", cache: Optional[str] = None, reps: int = 5):
    """Returns (Npad_y, Npad_x) and the general-kernel settings (a dict for
    Op.tune, empty for the 512 kernels or the defaults) for this grid and precision."""
    table: Dict[str, dict] = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    key = _key(grid, precision)
    if key in table and "tiles" in table[key]:
        return tuple(table[key]["npad"]), dict(table[key]["tiles"])
    timings, best_generic = {}, None
    for cand in candidates(grid, precision):
        ops = _setup(grid, mag, precision, cand)
        t = _time_ops(ops, reps)
        timings[f"{cand[0]}x{cand[1]}"] = t
        if ops[0].info.fast_path != 1 and (best_generic is None or t < best_generic[1]):
            best_generic = (cand, t)
        for op in ops:
            op.close()
    tiles, tuned_ms = {}, None
    if best_generic is not None:
        ops = _setup(grid, mag, precision, best_generic[0])
        tiles, tuned_ms = _refine(ops, reps, best_generic[1])
        for op in ops:
            op.close()
        timings[f"{best_generic[0][0]}x{best_generic[0][1]} tuned"] = tuned_ms
    best = min(timings, key=timings.get)
    npad = tuple(int(v) for v in best.split()[0].split("x"))
    if not best.endswith("tuned"):
        tiles = {}
    table[key] = {"npad": list(npad), "tiles": tiles, "ms_fwd_adj_both_fields": timings}
    if cache:
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return npad, tiles


def _time_pair(grid, mag, precision, npad, reps) -> float:
    ops = _setup(grid, mag, precision, npad)
    t = _time_ops(ops, reps)
    for op in ops:
        op.close()
    return t


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
