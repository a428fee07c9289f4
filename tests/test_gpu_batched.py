"""Batched form: several joint inversions of uneven sizes advanced by one CUDA
graph (gj_rrcg_batch_*), checked against the same solvers run one by one; and the
padded-size autotuner."""
import json

import numpy as np
import pytest
import torch

import synth
from tests.gpu_common import lib, rel

pytestmark = pytest.mark.gpu

SIZES = [(16, 16, 4), (12, 20, 3), (24, 24, 5), (32, 16, 4), (20, 20, 6)]


def make_problem(gj, nx, ny, nz, seed, npad=(0, 0), prec="fp32"):
    g = synth.uniform_grid(nx, ny, nx, ny, nz, 50.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    ops = [gj.bttb_setup(g, "gravity", precision=prec, npad=npad),
           gj.bttb_setup(g, "magnetic", mag, precision=prec, npad=npad)]
    dt = ops[0].dtype
    rng = np.random.default_rng(seed)
    mt = [torch.from_numpy(synth.dipping_blocks(g, v, seed, count=2)).to(dt).cuda() for v in (1.0, 0.1)]
    d = [ops[i].forward(mt[i]) for i in range(2)]
    sig = [0.01 * x.abs() + 0.01 * x.abs().max() for x in d]
    dob = [d[i] + sig[i] * torch.from_numpy(rng.standard_normal(g.s)).to(dt).cuda() for i in range(2)]
    wd = [torch.from_numpy(gj.depth_weights(g.z_edges, b)).to(dt).cuda() for b in (2.0, 3.0)]
    return g, ops, dob, sig, wd


def run(gj, batched, iters=12):
    params = gj.solver_params(p=(1, 1), lam=(2.0, 100.0), kmax=iters, stop_on_chi2=False)
    probs, solvers, models = [], [], []
    for i, (nx, ny, nz) in enumerate(SIZES):
        npad = (512, 512) if i == 2 else (0, 0)  # one problem on the specialised kernels
        g, ops, dob, sig, wd = make_problem(gj, nx, ny, nz, 10 + i, npad)
        m = [torch.zeros(g.n, device="cuda") for _ in range(2)]
        probs.append((ops, dob, sig, wd, m))
        solvers.append(gj.Solver(ops, params, dob, sig, wd, m))
        models.append(m)
    if batched:
        b = gj.Batch(solvers)
        b.step(iters)
        torch.cuda.synchronize()
        b.close()
    else:
        for s in solvers:
            s.iterate(iters, use_graph=True)
    reps = [s.report() for s in solvers]
    out = [[t.cpu().numpy().astype(np.float64) for t in m] for m in models]
    for s in solvers:
        s.close()
    return out, reps


def test_batched_graph_equals_one_by_one():
    gj = lib()
    ref, rref = run(gj, batched=False)
    got, rgot = run(gj, batched=True)
    for a, b, ra, rb in zip(got, ref, rgot, rref):
        assert ra["iterations"] == rb["iterations"] == 12
        for i in range(2):
            assert rel(a[i], b[i]) <= 1e-5


def test_autotuner_picks_a_valid_size_and_caches(tmp_path):
    gj = lib()
    from paper_2112_15562_gb300 import autotune

    g = synth.uniform_grid(40, 40, 40, 40, 6, 50.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    cache = str(tmp_path / "tune.json")
    npad = autotune.tune(g, mag, "fp32", cache=cache, reps=2)
    assert npad[0] >= 79 and npad[1] >= 79
    table = json.load(open(cache))
    (entry,) = table.values()
    assert tuple(entry["npad"]) == npad
    assert "512x512" in entry["ms_fwd_adj_both_fields"]
    assert autotune.tune(g, mag, "fp32", cache=cache) == npad  # served from the cache
    assert autotune.smooth_sizes(511, 3) == [512, 525, 540]
