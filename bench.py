#!/usr/bin/env python
"""Benchmark of the joint gravity-magnetic RRCG hot path on one or more GB300s.

Workload: 256x256 stations over 256x256x40 prisms of 100 m (2.6 M cells per model),
gravity and magnetic fields, Lp (p = 1) stabilisers and the Gramian coupling
(lambda = 2, 100), FP32 vectors and FFTs with FP64 scalars, padded BCCB size
512x512.  One step = one RRCG iteration (2 forward and 1 adjoint BTTB product per
field plus every fused vector update), replayed as one CUDA graph.  Inputs are
seeded and synthetic (three dipping blocks, 1 % noise).  The L2 cache is flushed
(256 MB write) before every timed step; each step is timed with CUDA events.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (a
bounded sample of the same workload, extrapolated to one iteration).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RRCG iters/s (joint gravity+magnetic, 256^2x40, FP32 vectors+FFTs, FP64 scalars)"
UNIT = "iters/s"
CONFIG = {"workload": "joint RRCG 256x256 stations x 256x256x40 prisms (100 m), p=1, lambda=(2,100), Npad 512x512",
          "cells_per_model": 256 * 256 * 40, "stations": 256 * 256, "fields": 2,
          "l2": "flushed before each timed step (256 MB write)", "inputs": "seeded synthetic (3 dipping blocks, 1% noise)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64, operator, e2e and CPU legs")
    ap.add_argument("--leg", choices=["c5", "fp64"], default=None,
                    help="time one leg alone at fixed padded sizes (no autotuning), for profiling: c5 = "
                         "512x512x48 forward + backward of both fields at 1024x1024; fp64 = the plain FP64 "
                         "iteration at 256x256x40, 512x512")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample

def _rows_worker(args):
    """Direct sums of the oracle for a chunk of forward rows and adjoint cells (one
    process of the pool); returns the seconds it took."""
    from oracle import operator as oop

    K, grid, m, r, stations, cells = args
    t0 = time.perf_counter()
    oop.forward_rows(K, grid, m, stations)
    oop.adjoint_cols(K, grid, r, cells)
    return time.perf_counter() - t0


def oracle_direct_all_cores(grid_full, mag, rows: int = 96, cols: int = 1536, layers: int = 4, seed: int = 0):
    """The oracle's direct sums (the plain definition of the products) on a pool of
    spawned processes, one per host core: ``rows`` forward rows over the top
    ``layers`` layers (scaled to nz; a row's cost is linear in the layer count) and
    ``cols`` adjoint cells per field, extrapolated to one RRCG iteration (2 forward
    and 1 adjoint products per field).  Returns (iters/s, seconds per iteration,
    processes, wall seconds)."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    import synth
    from oracle import operator as oop

    g = grid_full
    sub = synth.uniform_grid(g.sx, g.sy, g.nx, g.ny, layers, g.dx)
    sub.z_edges = g.z_edges[:layers + 1].copy()
    procs = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    jobs_rows, per_row, per_col = [], 0.0, 0.0
    with cf.ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(int, range(procs)))  # start the workers before timing
        wall = 0.0
        for f in (oop.GRAVITY, oop.MAGNETIC):
            K = oop.kernel_table(sub, f, mag)
            m = rng.uniform(0, 1, sub.n)
            r = rng.standard_normal(sub.s)
            st = np.array_split(rng.integers(0, sub.s, rows), procs)
            cl = np.array_split(rng.integers(0, sub.n, cols), procs)
            t0 = time.perf_counter()
            list(ex.map(_rows_worker, [(K, sub, m, r, st[k], np.array([], dtype=int)) for k in range(procs)]))
            t1 = time.perf_counter()
            list(ex.map(_rows_worker, [(K, sub, m, r, np.array([], dtype=int), cl[k]) for k in range(procs)]))
            t2 = time.perf_counter()
            per_row += (t1 - t0) / rows * (g.nz / layers)
            per_col += (t2 - t1) / cols
            wall += t2 - t0
    per_iter = 2 * g.s * per_row + g.n * per_col
    return 1.0 / per_iter, per_iter, procs, wall


def oracle_fft_iterations(w, iters: int, time_cap_s: float = 1e9, warmup: int = 0):
    """Whole RRCG iterations of the oracle at the full workload, with its FFT evaluation
    of the products (oracle.operator.BCCB, numpy FP64 on one core) and the same
    solver settings as the GPU leg; the tables are built first and not timed.
    Returns (seconds of each timed iteration, table seconds)."""
    import numpy as np
    from oracle import operator as oop
    from oracle import weights as owt
    from oracle.rrcg import RRCGParams, rrcg_joint

    g = w.grid
    t0 = time.perf_counter()
    B = [oop.BCCB(oop.kernel_table(g, oop.GRAVITY), g, 512, 512),
         oop.BCCB(oop.kernel_table(g, oop.MAGNETIC, w.mag), g, 512, 512)]
    t_tab = time.perf_counter() - t0
    obs = [owt.noisy_data(B[i].forward(w.m_true[i]), 0.01, 0.01, w.noise[i]) for i in range(2)]
    dob, sig = [o[0] for o in obs], [o[1] for o in obs]
    wst = [owt.depth_weight_cells(g.z_edges, b, g.nx, g.ny) for b in (2.0, 3.0)]
    stamps = []

    def fwd(i):
        def f(x):
            if i == 0:
                stamps.append(time.perf_counter())
            return B[i].forward(x)
        return f

    # one solve of kmax iterations; the forward of the gravity model opens each
    # iteration's timed span (the first, the residual of m_0, is setup)
    kmax = warmup + iters
    P = RRCGParams(p=(1, 1), alpha1=(2e4, 2e4), q=(0.95, 0.95), alpha_min=(5.0, 20.0), lam=(2.0, 100.0),
                   lo=(0.0, 0.0), hi=(1.0, 0.1), kmax=kmax, stop_on_chi2=False)
    t_start = time.perf_counter()

    class Capped(Exception):
        pass

    def fwd_capped(i):
        inner = fwd(i)

        def f(x):
            if i == 0 and time.perf_counter() - t_start > time_cap_s:
                raise Capped()
            return inner(x)
        return f

    try:
        rrcg_joint([fwd_capped(0), fwd_capped(1)], [B[0].adjoint, B[1].adjoint], dob, sig,
                   [np.zeros(g.n)] * 2, wst, P)
    except Capped:
        pass
    # gravity forwards per iteration: the residual of m_k and the product of p_k, so an
    # iteration spans two stamps
    starts = stamps[0::2]
    spans = [b - a for a, b in zip(starts[:-1], starts[1:])]
    return spans[warmup:], t_tab


def run_reference(args, rank):
    import synth

    if rank != 0:
        return
    w = synth.joint_256()
    t0 = time.perf_counter()
    spans, t_tab = oracle_fft_iterations(w, args.steps, time_cap_s=240.0, warmup=args.warmup)
    wall = time.perf_counter() - t0
    val = 1.0 / statistics.median(spans)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(spans), "warmup": args.warmup, "ms_per_step": 1e3 / val, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": CONFIG,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{len(spans)} whole RRCG iterations at 256x256x40 (of {args.steps} asked; "
                                       "240 s cap) by the oracle with its numpy-FFT FP64 evaluation of the products "
                                       f"(one core); tables {t_tab:.1f} s untimed; wall {wall:.1f} s"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------

def depth_weights(z_edges, beta: float):
    """The caller's depth weighting, an input of the solver: (z_c / z_c,top)^(-beta/2) at
    the layer centres (the Li & Oldenburg form, which the paper names without printing
    its exponent; the top layer has weight 1)."""
    import numpy as np

    z = np.asarray(z_edges, dtype=np.float64)
    zc = 0.5 * (z[:-1] + z[1:])
    return (zc / zc[0]) ** (-beta / 2.0)


def reduce_max_ms(total_ms: float, dist, device) -> float:
    """The timed region's length as the maximum over ranks (no-op on one rank)."""
    if dist is None:
        return total_ms
    import torch

    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, max_total_ms: float) -> float:
    """Iterations of all ranks (independent replicas) per second of the slowest rank."""
    return world * steps / (max_total_ms / 1e3)


def build_problem(gj, torch, prec, dev, npad=(0, 0), tiles=None):
    import numpy as np
    import synth

    w = synth.joint_256()
    g = w.grid
    ops = [gj.bttb_setup(g, "gravity", precision=prec, npad=npad),
           gj.bttb_setup(g, "magnetic", w.mag, precision=prec, npad=npad)]
    for o_ in ops:
        if tiles:
            o_.tune(**tiles)
    dt = ops[0].dtype
    m_true = [torch.from_numpy(x).to(dt).to(dev) for x in w.m_true]
    d_ex = [ops[i].forward(m_true[i]) for i in range(2)]
    sigma = [0.01 * d.abs() + 0.01 * d.abs().max() for d in d_ex]
    dobs = [d_ex[i] + sigma[i] * torch.from_numpy(w.noise[i]).to(dt).to(dev) for i in range(2)]
    wdep = [torch.from_numpy(depth_weights(g.z_edges, b)).to(dt).to(dev) for b in (2.0, 3.0)]
    return w, g, ops, dobs, sigma, wdep


def solver_for(gj, torch, ops, g, dobs, sigma, wdep, kmax, dev):
    m = [torch.zeros(g.n, dtype=ops[0].dtype, device=dev) for _ in range(2)]
    P = gj.solver_params(p=(1, 1), lam=(2.0, 100.0), alpha1=(2e4, 2e4), q=(0.95, 0.95), alpha_min=(5.0, 20.0),
                         lo=(0.0, 0.0), hi=(1.0, 0.1), kmax=kmax, stop_on_chi2=False)
    return gj.Solver(ops, P, dobs, sigma, wdep, m), m, P


def queued_times(torch, step, n, flush=None, skip=0):
    """Times ``n`` calls ``step(k)`` with a CUDA event pair each, all queued before the
    first is read back, so that the device never waits for the host inside a timed
    call; the L2 flush, when given, runs between the pairs.  Drops the first ``skip``."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        if flush is not None:
            flush.fill_(float(k))
        ev[k][0].record()
        step(k)
        ev[k][1].record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev][skip:]


def time_steps(torch, sv, steps, warmup, flush, profile=True, use_graph=True):
    for _ in range(warmup):
        flush.fill_(0.0)
        sv.iterate(1, use_graph=use_graph)
    torch.cuda.synchronize()
    if profile:
        sv.profile_read()
    times, pn, pms = [], 0, 0.0
    if not profile:
        return queued_times(torch, lambda k: sv.iterate(1, use_graph=use_graph), steps, flush), pn, pms
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for k in range(steps):
        flush.fill_(float(k))
        e0.record()
        sv.iterate(1, use_graph=use_graph)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        n, ms = sv.profile_read()
        pn += n
        pms += ms
    return times, pn, pms


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2112_15562_gb300 as gj

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

    w, g, ops, dobs, sigma, wdep = build_problem(gj, torch, "fp32", dev)
    kmax = 2 * (args.warmup + args.steps) + 8
    sv, m, P = solver_for(gj, torch, ops, g, dobs, sigma, wdep, kmax, dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    # region A (the headline): the whole iteration as one CUDA graph replay per step
    times, _, _ = time_steps(torch, sv, args.steps, args.warmup, flush, profile=False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    ck = clocks.stop()
    # region B: the same steps launched one by one (events inside a graph cannot be
    # timed), with CUDA events around every launch of the dominant kernel; the host
    # runs ahead of the device, so each pair brackets the kernel alone
    sv.profile(True)
    prof_mode = ("CUDA events on the launching stream around every launch, over a second timed region of "
                 f"{args.steps} steps launched one by one (the graph's launches, without the graph)")
    times_b, pn, pms = time_steps(torch, sv, args.steps, 2, flush, profile=True, use_graph=False)
    total_ms = reduce_max_ms(float(sum(times)), dist, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, args.steps, total_ms)
    rep = sv.report()
    sv.close()

    # roofline of the dominant kernel: the spectrum multiply-and-sum column pass
    o = ops[0].info
    kname = ("k_col_fwd512 (persistent layer-summed spectrum multiply + inverse column FFT, both fields)"
             if o.fast_path else "k_col_fwd_mac (layer-summed spectrum multiply, both fields)")
    traffic, traffic_note = profiled_traffic(o.fast_path)
    S_mag = o.nz * o.Ny * o.ncol * 8
    S_grav_min = even_spectrum_bytes(o, 4)
    alg_bytes_launch = S_mag + S_grav_min
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    avg_ms = pms / pn if pn else None
    achieved = alg_bytes_launch / (avg_ms * 1e-3) / 1e9 if avg_ms else None
    roof = {"kernel": kname, "bound": "hbm",
            "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm if achieved else None,
            "traffic": traffic, "traffic_source": traffic_note, "launches_timed": pn, "avg_launch_ms": avg_ms,
            "timing": prof_mode, "profiled_region_ms_per_step": float(sum(times_b)) / max(1, len(times_b)),
            "algorithmic_bytes_per_launch": alg_bytes_launch,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s"}
    n, s = g.n, g.s
    iter_alg = 3 * (S_mag + S_grav_min) + 2 * 36 * n + 6 * 4 * s * 2
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (f64 scalars)", "data": "synthetic", "config": dict(CONFIG),
            "roofline": roof, "clocks": ck, "gpu_launches": (10 if o.fast_path else 14) * args.steps,
            "iteration": {"algorithmic_bytes": iter_alg,
                          "algorithmic_GBs": iter_alg / (ms_per_step * 1e-3) / 1e9,
                          "frac_of_hbm": iter_alg / (ms_per_step * 1e-3) / 1e9 / hbm,
                          "wall_s": t_wall, "final_phi": rep["phi"], "S_G": rep["S_G"]}}
    if world > 1:
        line["config"]["parallelism"] = f"replicas x{world} (independent inversions, no collective)"

    if not args.no_extras and rank == 0:
        line["alu_peaks"] = alu_leg(gj, torch)
        line["roofline"]["alu"] = alu_fraction(o, avg_ms, line["alu_peaks"])
        line["operator"] = operator_leg(torch, ops, g, dev, flush, hbm)
        line["fp64"] = fp64_leg(gj, torch, dev, flush, value, hbm, line["alu_peaks"])
        line["p2"] = p2_leg(gj, torch, ops, g, dobs, sigma, wdep, dev, flush)
        line["operator_128"] = c2_leg(gj, torch, dev, flush, hbm)
        line["c5_512x48"] = c5_leg(gj, torch, dev, flush, hbm)
        line["e2e"] = e2e_leg(gj, torch, ops, g, dobs, sigma, wdep)
        line["batched"] = batched_leg(gj, torch, dev, flush)
        line["paper_shapes"] = paper_shapes_leg(gj, torch, dev, flush)
        if world == 1:
            spans, t_tab = oracle_fft_iterations(w, 2)
            v_all, per_all, procs, wall_all = oracle_direct_all_cores(w.grid, w.mag)
            c1 = oracle_c1_solve()
            line["cpu_baseline"] = {
                "value": 1.0 / statistics.median(spans), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"2 whole RRCG iterations at 256x256x40 by the oracle with its numpy-FFT FP64 evaluation "
                          f"of the products, one core (tables {t_tab:.1f} s, untimed)",
                "direct_sums_all_cores": {"value": v_all, "unit": UNIT, "cores": procs,
                                          "seconds_per_iteration": per_all, "wall_s": wall_all,
                                          "sample": "96 forward rows (top 4 layers, scaled to 40) and 1536 adjoint "
                                                    "cells per field by the oracle's direct sums on a spawned pool "
                                                    "of one process per core, extrapolated to one iteration"},
                "c1_dense_rrcg": c1}
    if rank == 0:
        print(json.dumps(line), flush=True)


def profiled_traffic(fast):
    """DRAM bytes per launch of the timed kernel from the committed ncu summary, if the
    kernel source is unchanged since that capture (else None)."""
    import hashlib
    import re

    if not fast:
        return None, "no capture for the generic kernel"
    src = os.path.join(ROOT, "paper_2112_15562_gb300", "csrc", "fast512.cuh")
    prof = os.path.join(ROOT, "profiles", "k_col_fwd512_joint256.md")
    try:
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
        txt = open(prof).read()
    except OSError:
        return None, "no ncu summary"
    m_hash = re.search(r"fast512\.cuh sha256: ([0-9a-f]{64})", txt)
    m_rd = re.search(r"dram__bytes_read\.sum: ([0-9.]+) MB", txt)
    m_wr = re.search(r"dram__bytes_write\.sum: ([0-9.]+) MB", txt)
    if not (m_hash and m_rd and m_wr):
        return None, "ncu summary incomplete"
    if m_hash.group(1) != digest:
        return None, "kernel changed since the ncu capture"
    return (float(m_rd.group(1)) + float(m_wr.group(1))) * 1e6, "profiles/k_col_fwd512_joint256.md (ncu, cold L2)"


def operator_leg(torch, ops, g, dev, flush, hbm, steps=50, elem=4):
    """G m + G^T r for both fields through gj_g_forward / gj_g_adjoint, in the ops'
    precision (elem bytes per real).  flush=None times warm (no L2 flush)."""
    dt = ops[0].dtype
    m = [torch.rand(g.n, device=dev, dtype=dt) for _ in range(2)]
    r = [torch.randn(g.s, device=dev, dtype=dt) for _ in range(2)]
    d = [torch.empty(g.s, device=dev, dtype=dt) for _ in range(2)]
    a = [torch.empty(g.n, device=dev, dtype=dt) for _ in range(2)]
    res = {}
    import paper_2112_15562_gb300 as gj

    for name in ("forward", "adjoint"):
        if name == "forward":
            call = lambda k: gj.g_forward_pair(ops, m, d)  # noqa: E731
        else:
            call = lambda k: gj.g_adjoint_pair(ops, r, a)  # noqa: E731
        res[name] = statistics.median(queued_times(torch, call, steps + 3, flush, skip=3))
    o = ops[0].info
    S_mag = o.nz * o.Ny * o.ncol * 2 * elem
    # per product: model and data vectors plus the layer spectra (the gravity spectrum
    # is real and even: its distinct values only)
    per_pair = 2 * (elem * g.n + elem * g.s) + S_mag + even_spectrum_bytes(o, elem)
    tot = res["forward"] + res["adjoint"]
    gbs = 2 * per_pair / (tot * 1e-3) / 1e9
    return {"forward_pair_ms": res["forward"], "adjoint_pair_ms": res["adjoint"],
            "algorithmic_bytes_fwd_plus_adj": 2 * per_pair, "algorithmic_GBs": gbs, "frac_of_hbm": gbs / hbm,
            "note": f"both fields per C-ABI call (gj_g_forward_pair / gj_g_adjoint_pair), "
                    f"{'L2 flushed' if flush is not None else 'warm'}, medians of {steps}"}


def fp64_leg(gj, torch, dev, flush, v32, hbm, alu, steps=8, warmup=2):
    """The plain FP64 form (every vector, spectrum and FFT in FP64, general kernels with
    the autotuned padded size, radix plan and tiles): the RRCG iteration and the
    standalone G m + G^T r of both fields."""
    import tempfile

    import synth
    from paper_2112_15562_gb300 import autotune

    wt = synth.joint_256()
    cache = os.path.join(tempfile.gettempdir(), "gj_autotune_bench.json")
    npad, tiles = autotune.tune_full(wt.grid, wt.mag, "fp64", cache=cache, reps=2)
    w, g, ops, dobs, sigma, wdep = build_problem(gj, torch, "fp64", dev, npad=npad, tiles=tiles)
    sv, m, P = solver_for(gj, torch, ops, g, dobs, sigma, wdep, steps + warmup + 2, dev)
    times, _, _ = time_steps(torch, sv, steps, warmup, flush, profile=False)
    sv.close()
    ms = sum(times) / steps
    opl = operator_leg(torch, ops, g, dev, flush, hbm, steps=10, elem=8)
    for o in ops:
        o.close()
    out = {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "fp32_speedup": v32 / (1e3 / ms), "dtype": "f64 (plain FP64 form)", "operator": opl,
           "npad_autotuned": list(npad), "tiles": tiles}
    # FFT flops of one iteration (5 N log2 N per complex 512-point transform, the
    # transforms of the generic kernels: row and column passes of 6 products)
    fl = iteration_fft_flops(g, N=max(npad))
    out["fft_GFLOPs_per_iteration"] = fl / 1e9
    if alu and alu.get("fp64_fma_tflops"):
        out["frac_of_fp64_fma_peak"] = fl / (ms * 1e-3) / 1e12 / alu["fp64_fma_tflops"]
    return out


def even_spectrum_bytes(o, elem):
    """Distinct values of the gravity spectrum: over stations that cover the prisms the
    table is even in both offsets, so its spectrum is real and even in kx and ky, and
    nz (Nx/2 + 1)(Ny/2 + 1) real values determine it."""
    return o.nz * o.ncol * (o.Ny // 2 + 1) * elem


def iteration_fft_flops(g, N=512):
    """5 N log2 N flops per complex N-point transform (the usual FFT count) over the
    transforms of one RRCG iteration on an N x N embedding: per field 2 forward
    products (rows: ny nz real lines, two per complex transform; columns: (N/2 + 1) nz
    transforms; one inverse column transform per column; sy/2 inverse row transforms)
    and 1 adjoint product (the reverse)."""
    import math

    f = 5 * N * math.log2(N)
    per_product = (g.ny * g.nz / 2 + (N // 2 + 1) * g.nz + (N // 2 + 1) + g.sy / 2) * f
    return 2 * 3 * per_product


def alu_leg(gj, torch):
    """FMA rates of the device (gj_probe_fma_rate), the compute roofline of the FFTs."""
    import ctypes as ct

    from paper_2112_15562_gb300 import _lib

    L = _lib.load()
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = {}
    for kind, key, iters in ((0, "fp32_fma_tflops", 4000), (1, "fp32x2_fma_tflops", 4000), (2, "fp64_fma_tflops", 500)):
        best = 0.0
        for _ in range(3):
            gf, ms = ct.c_double(), ct.c_double()
            _lib.check(L.gj_probe_fma_rate(kind, iters, ct.byref(gf), ct.byref(ms), st))
            best = max(best, gf.value / 1e3)
        out[key] = best
    out["note"] = ("gj_probe_fma_rate: 8 blocks of 256 threads per SM, 8 independent FMA chains per thread, "
                   "best of 3 launches timed with CUDA events at the clocks of the moment; 2 flops per FMA")
    return out


def alu_fraction(o, avg_ms, alu):
    """FFT flops of one launch of the dominant column kernel against the FP32 FMA rate:
    per field and layer (N/2 + 1) forward 512-point transforms and the spectrum
    multiply-adds, plus one inverse transform per column."""
    import math

    if not avg_ms or not alu.get("fp32_fma_tflops"):
        return None
    f = 5 * 512 * math.log2(512)
    cols = o.ncol
    fl = 2 * cols * o.nz * f + cols * o.nz * 512 * (8 + 4) + 2 * cols * f
    ach = fl / (avg_ms * 1e-3) / 1e12
    return {"flops_per_launch": fl, "achieved_tflops": ach, "fp32_fma_tflops": alu["fp32_fma_tflops"],
            "frac": ach / alu["fp32_fma_tflops"],
            "convention": "5 N log2 N per complex N-point transform; 8 (magnetic) and 4 (gravity, real spectrum) "
                          "flops per spectrum multiply-add"}


def p2_leg(gj, torch, ops, g, dobs, sigma, wdep, dev, flush, steps=20, warmup=3):
    """The same workload with the minimum-length stabiliser (p = 2, Sec. 3.1.5)."""
    m = [torch.zeros(g.n, dtype=ops[0].dtype, device=dev) for _ in range(2)]
    P = gj.solver_params(p=(2, 2), lam=(2.0, 100.0), alpha1=(2e4, 2e4), q=(0.95, 0.95), alpha_min=(5.0, 20.0),
                         lo=(0.0, 0.0), hi=(1.0, 0.1), kmax=steps + warmup + 2, stop_on_chi2=False)
    sv = gj.Solver(ops, P, dobs, sigma, wdep, m)
    times, _, _ = time_steps(torch, sv, steps, warmup, flush, profile=False)
    sv.close()
    ms = sum(times) / steps
    return {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "steps": steps, "p": [2, 2]}


def c2_leg(gj, torch, dev, flush, hbm, steps=20):
    """128x128 stations over 128x128x32 cells: G m + G^T r of both fields at the padded
    size 255 x 255 (3 x 5 x 17) and at the autotuned size, FP32 and FP64, with the L2
    flushed before every repetition (cold) and without (warm, the operator fits in L2)."""
    import tempfile

    import synth
    from paper_2112_15562_gb300 import autotune

    w = synth.operator_128()
    g = w.grid
    cache = os.path.join(tempfile.gettempdir(), "gj_autotune_bench.json")
    out = []
    for prec in ("fp32", "fp64"):
        auto, tiles = autotune.tune_full(g, w.mag, prec, cache=cache, reps=3)
        for npad in ((255, 255), tuple(auto)):
            ops = [gj.bttb_setup(g, "gravity", precision=prec, npad=npad),
                   gj.bttb_setup(g, "magnetic", w.mag, precision=prec, npad=npad)]
            tuned = tuple(npad) == tuple(auto)
            for o_ in ops:
                if tuned and tiles:
                    o_.tune(**tiles)
            res = {"precision": prec, "npad": list(npad), "autotuned": tuned, "tiles": tiles if tuned else {},
                   "fast_path": bool(ops[0].info.fast_path)}
            for mode in ("cold", "warm"):
                opl = operator_leg(torch, ops, g, dev, flush if mode == "cold" else None, hbm, steps=steps,
                                   elem=8 if prec == "fp64" else 4)
                res[mode] = {k: opl[k] for k in ("forward_pair_ms", "adjoint_pair_ms", "algorithmic_GBs",
                                                 "frac_of_hbm")}
            out.append(res)
            for o in ops:
                o.close()
    return {"runs": out, "note": "both fields, standalone C-ABI calls, medians; algorithmic bytes as for the "
                                 "256x256x40 line (spectrum bytes at the padded size in use)"}


def c5_step(gj, ops, m, gd):
    """One forward + backward of both fields through torch.autograd; the gradients are
    cleared first, as an optimiser's zero_grad(set_to_none=True) does, so that no
    accumulation kernel runs."""
    for t in m:
        t.grad = None
    for i in range(2):
        gj.G(ops[i], m[i]).backward(gd[i])


def c5_graph(gj, torch, ops, m, gd, steps, flush, alg, hbm):
    """The same forward + backward step captured once in a CUDA graph (torch.cuda.graph;
    the library's products launch on the capturing stream) and replayed, so that the
    step's time is the device's and not the host's issue of the autograd step; the
    replayed gradients are compared with an eager step's."""
    c5_step(gj, ops, m, gd)
    ref = [t.grad.clone() for t in m]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            c5_step(gj, ops, m, gd)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        c5_step(gj, ops, m, gd)
    graph.replay()
    torch.cuda.synchronize()
    err = max(float((t.grad - r).norm() / r.norm()) for t, r in zip(m, ref))
    ts = queued_times(torch, lambda k: graph.replay(), steps + 1, flush, skip=1)
    ms = statistics.median(ts)
    del graph
    return {"ms_per_fwd_bwd_both_fields": ms, "algorithmic_GBs": alg / (ms * 1e-3) / 1e9,
            "frac_of_hbm": alg / (ms * 1e-3) / 1e9 / hbm, "grad_rel_diff_vs_eager": err}


def c5_leg(gj, torch, dev, flush, hbm):
    """512x512 stations over 512x512x48 cells of 100 m (12.6 M cells per model), FP32,
    padded 1024 x 1024: forward plus backward (G m through torch.autograd, backward =
    the adjoint product) of both fields, with the layer spectra stored and with every
    layer's spectrum rebuilt from the closed forms inside each product."""
    import synth

    import tempfile

    from paper_2112_15562_gb300 import autotune

    g = synth.uniform_grid(512, 512, 512, 512, 48, 100.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    cache = os.path.join(tempfile.gettempdir(), "gj_autotune_bench.json")
    npad, tiles = autotune.tune_full(g, mag, "fp32", cache=cache, reps=2)
    out = {"workload": "fwd+bwd of both fields at 512x512x48, FP32, L2 flushed per step",
           "npad_autotuned": list(npad), "tiles": tiles}
    for mode, steps in (("stored", 5), ("recomputed", 2)):
        t0 = time.perf_counter()
        ops = [gj.bttb_setup(g, "gravity", precision="fp32", npad=npad, recompute=mode == "recomputed"),
               gj.bttb_setup(g, "magnetic", mag, precision="fp32", npad=npad, recompute=mode == "recomputed")]
        for o_ in ops:
            if tiles:
                o_.tune(**tiles)
        t_setup = time.perf_counter() - t0
        m = [torch.rand(g.n, device=dev, requires_grad=True) for _ in range(2)]
        gd = [torch.randn(g.s, device=dev) for _ in range(2)]
        ts = queued_times(torch, lambda k: c5_step(gj, ops, m, gd), steps + 1, flush, skip=1)
        ms = statistics.median(ts)
        o = ops[0].info
        S_mag = o.nz * o.Ny * o.ncol * 8
        alg = 2 * 2 * (4 * g.n + 4 * g.s) + 2 * (S_mag + even_spectrum_bytes(o, 4))
        res = {"ms_per_fwd_bwd_both_fields": ms, "setup_s": t_setup, "steps": steps,
               "spectrum_bytes_both_fields": ops[0].info.spectrum_bytes + ops[1].info.spectrum_bytes,
               "cells_per_s": 2 * g.n / (ms * 1e-3)}
        if mode == "stored":
            res["algorithmic_GBs"] = alg / (ms * 1e-3) / 1e9
            res["frac_of_hbm"] = res["algorithmic_GBs"] / hbm
            try:
                res["graph"] = c5_graph(gj, torch, ops, m, gd, steps, flush, alg, hbm)
            except Exception as exc:  # capture refused: the eager figure stands alone
                torch.cuda.synchronize()
                res["graph"] = {"unavailable": f"{type(exc).__name__}: {exc}"[:200]}
        out[mode] = res
        for op in ops:
            op.close()
        del m, gd
        torch.cuda.empty_cache()
    return out


def oracle_c1_solve():
    """The oracle's full FP64 dense joint RRCG on the 16x16x8 workload (50 iterations,
    chi^2 stop off), timed end to end on one core, matrices included."""
    import numpy as np
    import synth
    from oracle import operator as oop
    from oracle import weights as owt
    from oracle.rrcg import RRCGParams, rrcg_joint

    t0 = time.perf_counter()
    w = synth.small_joint()
    g = w.grid
    A = [oop.dense_matrix(g, oop.GRAVITY), oop.dense_matrix(g, oop.MAGNETIC, w.mag)]
    obs = [owt.noisy_data(A[i] @ w.m_true[i], 0.01, 0.01, w.noise[i]) for i in range(2)]
    wst = [owt.depth_weight_cells(g.z_edges, b, g.nx, g.ny) for b in (2.0, 3.0)]
    t1 = time.perf_counter()
    P = RRCGParams(p=(1, 1), lam=(50.0, 1500.0), kmax=50, stop_on_chi2=False)
    rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)], [lambda y, i=i: A[i].T @ y for i in range(2)],
               [o[0] for o in obs], [o[1] for o in obs], [np.zeros(g.n)] * 2, wst, P)
    t2 = time.perf_counter()
    return {"seconds_total": t2 - t0, "seconds_solve": t2 - t1, "iterations": 50,
            "iters_per_s": 50 / (t2 - t1), "cores": 1, "workload": "joint 16x16x8, FP64 dense, p=1, lambda=(50,1500)"}


def batched_leg(gj, torch, dev, flush, steps=20, warmup=3):
    """Sixteen independent joint inversions of uneven sizes (64..256 per side,
    16..40 layers, seeded) advanced together by one CUDA graph per step; padded
    sizes chosen by the autotuner.  Value: total iterations per second."""
    import tempfile

    import numpy as np
    import synth
    from paper_2112_15562_gb300 import autotune

    cache = os.path.join(tempfile.gettempdir(), "gj_autotune_bench.json")
    sizes = synth.batched_sizes()
    solvers, keep, npads, cells = [], [], [], 0
    for i, (nx, ny, nz) in enumerate(sizes):
        gr = synth.uniform_grid(nx, ny, nx, ny, nz, 100.0)
        mag = synth.Mag(50000.0, 60.0, 10.0)
        npad, tiles = autotune.tune_full(gr, mag, "fp32", cache=cache, reps=3)
        npads.append(list(npad) + ([tiles] if tiles else []))
        ops = [gj.bttb_setup(gr, "gravity", precision="fp32", npad=npad),
               gj.bttb_setup(gr, "magnetic", mag, precision="fp32", npad=npad)]
        for o_ in ops:
            if tiles:
                o_.tune(**tiles)
        mt = [torch.from_numpy(synth.dipping_blocks(gr, v, 40 + i)).float().to(dev) for v in (1.0, 0.1)]
        d = [ops[k].forward(mt[k]) for k in range(2)]
        sig = [0.01 * x.abs() + 0.01 * x.abs().max() for x in d]
        rng = np.random.default_rng(40 + i)
        dob = [d[k] + sig[k] * torch.from_numpy(rng.standard_normal(gr.s)).float().to(dev) for k in range(2)]
        wd = [torch.from_numpy(depth_weights(gr.z_edges, b)).float().to(dev) for b in (2.0, 3.0)]
        m = [torch.zeros(gr.n, device=dev) for _ in range(2)]
        P = gj.solver_params(p=(1, 1), lam=(2.0, 100.0), kmax=steps + warmup + 4, stop_on_chi2=False)
        solvers.append(gj.Solver(ops, P, dob, sig, wd, m))
        keep.append((ops, dob, sig, wd, m))
        cells += 2 * gr.n
    batch = gj.Batch(solvers)
    for _ in range(warmup):
        batch.step(1)
    torch.cuda.synchronize()
    ts = queued_times(torch, lambda k: batch.step(1), steps, flush)
    batch.close()
    for s_ in solvers:
        s_.close()
    ms = sum(ts) / steps
    return {"value": len(sizes) * 1e3 / ms, "unit": "problem-iters/s", "ms_per_step": ms, "problems": len(sizes),
            "sizes_nx_ny_nz": [list(x) for x in sizes], "npad_autotuned": npads, "cells_both_fields": cells,
            "note": "one graph replay advances all 16 inversions by one RRCG iteration; L2 flushed per step"}


# the paper's workloads (Secs. 3.1, 3.2, 4): shape, cell sizes, and the laptop's
# seconds per iteration (total time / iterations as printed), for context only
PAPER_SHAPES = [
    ("two cubes 50x30x10 (Sec. 3.1.2)", (50, 30, 10), (100.0, 100.0), 45.0 / 52),
    ("five bodies 150x100x10 (Sec. 3.2)", (150, 100, 10), (100.0, 100.0), 4872.0 / 96),
    ("field data 146x148x20 (Sec. 4)", (146, 148, 20), (250.0, 500.0), 20 * 3600.0 / 186),
]


def paper_shapes_leg(gj, torch, dev, flush, steps=20, warmup=3):
    """Seconds per RRCG iteration on seeded stand-ins with the shapes of the paper's
    three workloads (the bodies and field data themselves are not available), FP32
    with autotuned padding, next to the paper's laptop figures."""
    import tempfile

    import numpy as np
    import synth
    from paper_2112_15562_gb300 import autotune

    cache = os.path.join(tempfile.gettempdir(), "gj_autotune_bench.json")
    out = []
    for name, (nx, ny, nz), (dh, dz), laptop in PAPER_SHAPES:
        gr = synth.uniform_grid(nx, ny, nx, ny, nz, dh, dz=dz)
        mag = synth.Mag(50000.0, 45.0, 45.0)
        npad, tiles = autotune.tune_full(gr, mag, "fp32", cache=cache, reps=3)
        ops = [gj.bttb_setup(gr, "gravity", precision="fp32", npad=npad),
               gj.bttb_setup(gr, "magnetic", mag, precision="fp32", npad=npad)]
        for o_ in ops:
            if tiles:
                o_.tune(**tiles)
        mt = [torch.from_numpy(synth.dipping_blocks(gr, v, 7)).float().to(dev) for v in (1.0, 0.1)]
        d = [ops[k].forward(mt[k]) for k in range(2)]
        sig = [0.01 * x.abs() + 0.01 * x.abs().max() for x in d]
        rng = np.random.default_rng(7)
        dob = [d[k] + sig[k] * torch.from_numpy(rng.standard_normal(gr.s)).float().to(dev) for k in range(2)]
        wd = [torch.from_numpy(depth_weights(gr.z_edges, b)).float().to(dev) for b in (2.0, 3.0)]
        sv, m, P = solver_for(gj, torch, ops, gr, dob, sig, wd, steps + warmup + 4, dev)
        ts, _, _ = time_steps(torch, sv, steps, warmup, flush, profile=False)
        sv.close()
        s_it = sum(ts) / steps / 1e3
        out.append({"workload": name, "npad": list(npad), "tiles": tiles, "s_per_iter": s_it, "laptop_s_per_iter": laptop,
                    "ratio_vs_laptop": laptop / s_it})
    return {"runs": out, "note": "laptop figures: the paper's Intel i7-10750H, FP64, total time / iterations; "
                                 "a different machine and workload (context, not a target)"}


def e2e_leg(gj, torch, ops, g, dobs, sigma, wdep, iters=50, calls=3):
    """The host-buffer solve through the C ABI (gj_rrcg_joint_solve_host): page-locked
    host inputs are copied in by the library, the solver is created (graph capture
    included), ``iters`` iterations (the workload's 50) run and both models are copied
    back; timed on the wall clock around each call, the median of ``calls`` calls."""
    host = [x.cpu().pin_memory() for x in list(dobs) + list(sigma) + list(wdep)]
    m0 = [torch.zeros(g.n, dtype=ops[0].dtype).pin_memory() for _ in range(2)]
    P = gj.solver_params(p=(1, 1), lam=(2.0, 100.0), alpha1=(2e4, 2e4), q=(0.95, 0.95), alpha_min=(5.0, 20.0),
                         lo=(0.0, 0.0), hi=(1.0, 0.1), kmax=iters, stop_on_chi2=False)
    gj.rrcg_joint_solve_host(ops, P, host[0:2], host[2:4], host[4:6], m0)  # warm-up
    for t in m0:
        t.zero_()
    spans = []
    for _ in range(calls):
        for t in m0:
            t.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = gj.rrcg_joint_solve_host(ops, P, host[0:2], host[2:4], host[4:6], m0)
        spans.append(time.perf_counter() - t0)
    dt = statistics.median(spans)
    return {"value": iters / dt, "unit": UNIT, "h2d_bytes_per_step": rep["h2d_bytes"] / iters,
            "d2h_bytes_per_step": rep["d2h_bytes"] / iters, "iterations_per_call": iters, "call_s": dt,
            "calls_s": spans,
            "note": "gj_rrcg_joint_solve_host (C ABI, host buffers): H2D of data, sigma, depth weights and start "
                    "models from page-locked memory, solver creation and graph capture, the iterations, D2H of "
                    "both models"}


def run_leg(args):
    """One leg alone, at fixed padded sizes, ``--steps`` timed steps after ``--warmup``
    (the launch lists of ``profiles/`` come from these runs)."""
    import torch

    import paper_2112_15562_gb300 as gj

    dev = torch.device("cuda:0")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    if args.leg == "fp64":
        w, g, ops, dobs, sigma, wdep = build_problem(gj, torch, "fp64", dev, npad=(512, 512))
        sv, m, P = solver_for(gj, torch, ops, g, dobs, sigma, wdep, args.steps + args.warmup + 2, dev)
        times, _, _ = time_steps(torch, sv, args.steps, args.warmup, flush, profile=False)
        sv.close()
        print(json.dumps({"leg": "fp64 joint RRCG 256x256x40, Npad 512x512", "ms_per_iteration": sum(times) / len(times),
                          "steps": args.steps}))
        return
    import synth

    g = synth.uniform_grid(512, 512, 512, 512, 48, 100.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    ops = [gj.bttb_setup(g, "gravity", precision="fp32", npad=(1024, 1024)),
           gj.bttb_setup(g, "magnetic", mag, precision="fp32", npad=(1024, 1024))]
    m = [torch.rand(g.n, device=dev, requires_grad=True) for _ in range(2)]
    gd = [torch.randn(g.s, device=dev) for _ in range(2)]
    ts = queued_times(torch, lambda k: c5_step(gj, ops, m, gd), args.warmup + args.steps, flush, skip=args.warmup)
    print(json.dumps({"leg": "512x512x48 fwd+bwd of both fields, Npad 1024x1024, FP32",
                      "ms_per_fwd_bwd_both_fields": statistics.median(ts), "steps": args.steps}))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.leg:
        run_leg(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
