"""Batched form: several joint inversions of uneven sizes advanced by one CUDA
graph (gj_rrcg_batch_*), checked against the same solvers run one by one; and the
padded-size autotuner."""
import json

import numpy as np
import pytest
import torch

import synth
from oracle import weights as owt
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
    wd = [torch.from_numpy(owt.depth_weights(g.z_edges, b)).to(dt).cuda() for b in (2.0, 3.0)]
    return g, ops, dob, sig, wd


def run(gj, batched, iters=12):
    params = gj.solver_params(p=(1, 1), lam=(2.0, 100.0), kmax=iters, stop_on_chi2=False)
    probs, solvers, models = [], [], []
    for i, (nx, ny, nz) in enumerate(SIZES):
        # one problem on each of the specialised kernels' padded sizes
        npad = {1: (1024, 24), 2: (512, 512), 4: (256, 512)}.get(i, (0, 0))
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


def test_batched_problem_matches_oracle():
    """One problem of a batch (16x16x6 on the 512 kernels, data from the dense oracle)
    against the FP64 oracle's RRCG, while two other problems of different sizes run in
    the same graph (Eq. RRCG:1-8); the batch gives each fast-path solver a share of
    the SMs, so the branches run concurrently."""
    from oracle import operator as oop
    from oracle.rrcg import RRCGParams, rrcg_joint

    gj = lib()
    g = synth.uniform_grid(16, 16, 16, 16, 6, 50.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    A = [oop.dense_matrix(g, oop.GRAVITY), oop.dense_matrix(g, oop.MAGNETIC, mag)]
    mt = [synth.dipping_blocks(g, v, 91, count=2) for v in (1.0, 0.1)]
    e = synth.standard_normal((2, g.s), 92)
    obs = [owt.noisy_data(A[i] @ mt[i], 0.01, 0.01, e[i]) for i in range(2)]
    dob, sig = [o[0] for o in obs], [o[1] for o in obs]
    wdep = [owt.depth_weights(g.z_edges, b) for b in (2.0, 3.0)]
    kw = dict(p=(1, 1), lam=(2.0, 100.0), kmax=12, stop_on_chi2=False)
    ref = rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)], [lambda y, i=i: A[i].T @ y for i in range(2)],
                     dob, sig, [np.zeros(g.n)] * 2, [np.repeat(wdep[i], g.nx * g.ny) for i in range(2)],
                     RRCGParams(**kw))
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).float().cuda()
    ops = [gj.bttb_setup(g, "gravity", precision="fp32", npad=(512, 512)),
           gj.bttb_setup(g, "magnetic", mag, precision="fp32", npad=(512, 512))]
    m = [torch.zeros(g.n, device="cuda") for _ in range(2)]
    solvers = [gj.Solver(ops, gj.solver_params(**kw), [dev(x) for x in dob], [dev(x) for x in sig],
                         [dev(x) for x in wdep], m, history=True)]
    others = []
    for i, (nx, ny, nz) in enumerate([(24, 20, 5), (40, 40, 8)]):
        go, opso, dobo, sigo, wdo = make_problem(gj, nx, ny, nz, 60 + i, npad=[(256, 512), (512, 512)][i])
        mo = [torch.zeros(go.n, device="cuda") for _ in range(2)]
        others.append((opso, dobo, sigo, wdo, mo))
        solvers.append(gj.Solver(opso, gj.solver_params(**kw), dobo, sigo, wdo, mo))
    b = gj.Batch(solvers)
    b.step(12)
    torch.cuda.synchronize()
    b.close()
    rep = solvers[0].report()
    assert rep["iterations"] == 12
    for k in range(13):
        for i in range(2):
            assert rep["history"][k]["phi"][i] == pytest.approx(ref.history[k]["phi"][i], rel=1e-4), (k, i)
    for i in range(2):
        assert rel(m[i].double().cpu().numpy(), ref.m[i]) <= 1e-3
    for s_ in solvers:
        s_.close()


def test_op_tune_keeps_the_product():
    """gj_op_tune (tiles and radix plan of the general kernels) changes only rounding."""
    gj = lib()
    g = synth.uniform_grid(20, 18, 20, 18, 4, 50.0)
    from oracle import operator as oop

    A = oop.dense_matrix(g, oop.MAGNETIC, synth.Mag(50000.0, 60.0, 10.0))
    op = gj.bttb_setup(g, "magnetic", synth.Mag(50000.0, 60.0, 10.0), precision="fp64", npad=(40, 42))
    m = np.random.default_rng(1).standard_normal(g.n)
    for kw in ({}, {"P_row": 2}, {"C_col": 1}, {"L_grp": 1}, {"radix_order": 1}, {"radix_order": 2},
               {"P_row": 16, "C_col": 16, "L_grp": 4, "radix_order": 0}):
        op.tune(**kw)
        for k, v in kw.items():
            assert op.tiles()[k] == v
        d = op.forward(torch.from_numpy(m).cuda()).cpu().numpy()
        assert rel(d, A @ m) <= 1e-10, kw
    with pytest.raises(gj.GJError):
        op.tune(P_row=4096)
    with pytest.raises(gj.GJError):
        op.tune(radix_order=7)


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
    # the full search on FP64 (general kernels only): size, radix plan and tiles
    npad64, tiles = autotune.tune_full(g, mag, "fp64", cache=cache, reps=2)
    assert npad64[0] >= 79 and npad64[1] >= 79
    assert set(tiles) <= set(autotune.KNOBS) and all(v in autotune.KNOBS[k] for k, v in tiles.items())
    entry = json.load(open(cache))[autotune._key(g, "fp64")]
    assert any(k.endswith("tuned") for k in entry["ms_fwd_adj_both_fields"])
    assert autotune.tune_full(g, mag, "fp64", cache=cache) == (npad64, tiles)


def test_lambda_sweep_matches_single_solves():
    gj = lib()
    g, ops, dob, sig, wd = make_problem(gj, 16, 16, 6, 77)
    lambdas = [(0.0, 0.0), (2.0, 100.0), (50.0, 1500.0)]
    kw = dict(p=(1, 1), kmax=15, stop_on_chi2=False)
    out = gj.lambda_sweep(g, synth.Mag(50000.0, 60.0, 10.0), dob, sig, wd, lambdas, precision="fp32", **kw)
    assert len(out["runs"]) == 3
    for lam, run in zip(lambdas, out["runs"]):
        opsi = [gj.bttb_setup(g, "gravity", precision="fp32"),
                gj.bttb_setup(g, "magnetic", synth.Mag(50000.0, 60.0, 10.0), precision="fp32")]
        m = [torch.zeros(g.n, device="cuda") for _ in range(2)]
        gj.rrcg_joint_solve(opsi, gj.solver_params(lam=lam, **kw), dob, sig, wd, m)
        for i in range(2):
            assert rel(run["models"][i], m[i].double().cpu().numpy()) <= 1e-5
        assert run["iterations"] == 15
        assert -1.0 <= run["pearson"] <= 1.0
    # with the stop test off nothing "converges": no pair qualifies
    assert out["selected"] is None


def test_lambda_sweep_selects_the_pair_the_oracle_selects():
    """The selection of Secs. 3.1.3 and 5 with the chi^2 stop on (Eq. chi2): the sweep
    keeps the smallest (lambda1, lambda2) whose solve fits both data sets and whose
    models correlate above the threshold.  The same pairs run through the FP64 oracle
    on the same host-made data decide which pair that is; here lambda = 0 fits but
    correlates below 0.96, (1, 50) fits and correlates, and (5, 300) does not fit
    within kmax."""
    from oracle.rrcg import RRCGParams, rrcg_joint
    from oracle import operator as oop

    gj = lib()
    g = synth.uniform_grid(16, 16, 16, 16, 6, 50.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    A = [oop.dense_matrix(g, oop.GRAVITY), oop.dense_matrix(g, oop.MAGNETIC, mag)]
    mt = [synth.dipping_blocks(g, v, 77, count=2) for v in (1.0, 0.1)]
    e = synth.standard_normal((2, g.s), 78)
    obs = [owt.noisy_data(A[i] @ mt[i], 0.01, 0.01, e[i]) for i in range(2)]
    dob, sig = [o[0] for o in obs], [o[1] for o in obs]
    wdep = [owt.depth_weights(g.z_edges, b) for b in (2.0, 3.0)]
    lambdas = [(0.0, 0.0), (1.0, 50.0), (5.0, 300.0)]
    kw = dict(p=(1, 1), alpha1=(100.0, 100.0), q=(0.85, 0.85), lo=(0.0, 0.0), hi=(1.0, 0.1), kmax=250,
              stop_on_chi2=True)
    thr = 0.96
    want = []
    for lam in lambdas:
        r = rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)], [lambda y, i=i: A[i].T @ y for i in range(2)],
                       dob, sig, [np.zeros(g.n)] * 2, [np.repeat(wdep[i], g.nx * g.ny) for i in range(2)],
                       RRCGParams(lam=lam, **kw))
        want.append((r.converged, float(np.corrcoef(r.m[0], r.m[1])[0, 1])))
    expect = next(i for i, (c, pc) in enumerate(want) if c and pc >= thr)
    assert expect == 1 and want[0][0] and want[0][1] < thr and not want[2][0]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).float().cuda()
    out = gj.lambda_sweep(g, mag, [dev(x) for x in dob], [dev(x) for x in sig], [dev(x) for x in wdep], lambdas,
                          precision="fp32", corr_threshold=thr, **kw)
    assert out["selected"] == expect
    for run, (conv, pc) in zip(out["runs"], want):
        assert run["converged"] == conv
        # a run that stops on chi^2 may stop an iteration earlier or later in FP32
        assert run["pearson"] == pytest.approx(pc, abs=0.02)
    assert abs(gj.pearson(np.arange(5.0), 2 * np.arange(5.0) + 1) - 1.0) < 1e-12
