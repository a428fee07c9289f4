"""Parity of the CUDA joint RRCG solve (gj_rrcg_joint_solve, Eq. RRCG:1-8,
Secs. 2.5, 2.6, 2.8) with the FP64 oracle, iteration by iteration."""
import numpy as np
import pytest
import torch

import synth
from oracle import operator as oop
from oracle import weights as owt
from oracle.rrcg import RRCGParams, rrcg_joint
from tests.gpu_common import lib, rel, to_dev

pytestmark = pytest.mark.gpu


def joint_case(w):
    g = w.grid
    A = [oop.dense_matrix(g, oop.GRAVITY), oop.dense_matrix(g, oop.MAGNETIC, w.mag)]
    d_ex = [A[i] @ w.m_true[i] for i in range(2)]
    obs = [owt.noisy_data(d_ex[i], *w.tau[i], w.noise[i]) for i in range(2)]
    dob = [o[0] for o in obs]
    sig = [o[1] for o in obs]
    wdep = [owt.depth_weights(g.z_edges, 2.0), owt.depth_weights(g.z_edges, 3.0)]
    return g, A, dob, sig, wdep


def run_oracle(g, A, dob, sig, wdep, P, m0=None, m_apr=None, w_hard=None):
    m0 = [np.zeros(g.n)] * 2 if m0 is None else m0
    w_static = [np.repeat(wdep[i], g.nx * g.ny) * (1.0 if w_hard is None else w_hard[i]) for i in range(2)]
    return rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)], [lambda y, i=i: A[i].T @ y for i in range(2)],
                      dob, sig, m0, w_static, P, m_apr=m_apr)


def run_gpu(gj, w, g, dob, sig, wdep, prec, kw, m0=None, graph=None, npad=(0, 0), m_apr=None, w_hard=None):
    ops = [gj.bttb_setup(g, "gravity", precision=prec, npad=npad),
           gj.bttb_setup(g, "magnetic", w.mag, precision=prec, npad=npad)]
    m = [to_dev(np.zeros(g.n) if m0 is None else m0[i], prec) for i in range(2)]
    args = ([to_dev(x, prec) for x in dob], [to_dev(x, prec) for x in sig], [to_dev(x, prec) for x in wdep], m)
    P = gj.solver_params(**kw)
    if m_apr is not None or w_hard is not None:
        opt = dict(m_apr=None if m_apr is None else [to_dev(x, prec) for x in m_apr],
                   w_hard=None if w_hard is None else [to_dev(x, prec) for x in w_hard])
        rep = gj.rrcg_joint_solve(ops, P, *args, history=True, **opt)
        return [t.cpu().numpy().astype(np.float64) for t in m], rep
    if graph is None:
        rep = gj.rrcg_joint_solve(ops, P, *args, history=True)
    else:
        sv = gj.Solver(ops, P, *args, history=True)
        left = kw["kmax"]
        while left > 0 and not sv.done():
            sv.iterate(min(5, left), use_graph=graph)
            left -= 5
        rep = sv.report()
        sv.close()
    return [t.cpu().numpy().astype(np.float64) for t in m], rep


KW = dict(p=(1, 1), alpha1=(2e4, 2e4), q=(0.95, 0.95), lam=(50.0, 1500.0), lo=(0.0, 0.0), hi=(1.0, 0.1),
          kmax=50, stop_on_chi2=False)


def oracle_params(kw):
    return RRCGParams(p=kw["p"], alpha1=kw["alpha1"], q=kw["q"], alpha_min=kw.get("alpha_min", (0.0, 0.0)),
                      lam=kw["lam"], lo=kw["lo"], hi=kw["hi"], kmax=kw["kmax"], stop_on_chi2=kw["stop_on_chi2"],
                      scalars=kw.get("scalars", "auto"), anchor=kw.get("anchor", "apriori"),
                      gramian_space=kw.get("gramian_space", "original"))


@pytest.fixture(scope="module")
def small():
    w = synth.small_joint()
    return (w,) + joint_case(w)


def compare_history(hg, ho, tol):
    assert len(hg) == len(ho)
    for k, (a, b) in enumerate(zip(hg, ho)):
        for i in range(2):
            assert a["phi"][i] == pytest.approx(b["phi"][i], rel=tol), (k, "phi", i)
            assert a["alpha"][i] == pytest.approx(b["alpha"][i], rel=1e-14), (k, "alpha", i)
            if "s" in b:
                assert a["s"][i] == pytest.approx(b["s"][i], rel=tol), (k, "s", i)
                assert a["beta"][i] == pytest.approx(b["beta"][i], rel=tol, abs=1e-300), (k, "beta", i)


def test_joint_fp64_matches_oracle_step_by_step(small):
    gj = lib()
    w, g, A, dob, sig, wdep = small
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(KW))
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, "fp64", KW)
    assert rep["iterations"] == ref.iterations == 50
    compare_history(rep["history"], ref.history, 1e-9)
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= 1e-9
        assert m[i].min() >= KW["lo"][i] and m[i].max() <= KW["hi"][i]


def test_joint_fp32_mixed_within_model_tolerance(small):
    gj = lib()
    w, g, A, dob, sig, wdep = small
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(KW))
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, "fp32", KW)
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= 1e-3, (i, rel(m[i], ref.m[i]))


@pytest.mark.parametrize("variant", ["per_field_lam0", "p2_joint", "alpha_floor_stop", "weighted_gramian",
                                     "previous_anchor"])
def test_solver_variants_fp64(small, variant):
    gj = lib()
    w, g, A, dob, sig, wdep = small
    kw = dict(KW)
    if variant == "per_field_lam0":
        kw.update(lam=(0.0, 0.0), kmax=30)
    elif variant == "p2_joint":
        kw.update(p=(2, 2), lam=(50.0, 8e5), alpha1=(2e4, 4e4), alpha_min=(50.0, 50.0), kmax=40)
    elif variant == "weighted_gramian":  # Sec. 3.1.4: Eq. steepestascenta/b on W m
        kw.update(lam=(5000.0, 10000.0), gramian_space="weighted", kmax=40)
    elif variant == "previous_anchor":  # RRCG:4 with the printed m~_k - m~_{k-1}
        kw.update(anchor="previous", kmax=30)
    else:
        kw.update(alpha_min=(500.0, 900.0), q=(0.8, 0.85), kmax=150, stop_on_chi2=True)
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(kw))
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, "fp64", kw)
    assert rep["iterations"] == ref.iterations
    assert rep["converged"] == ref.converged
    compare_history(rep["history"], ref.history, 1e-8)
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= 1e-8


@pytest.mark.parametrize("graph", [False, True])
def test_stepwise_graph_and_eager_match_one_shot(small, graph):
    gj = lib()
    w, g, A, dob, sig, wdep = small
    kw = dict(KW, kmax=12)
    m1, r1 = run_gpu(gj, w, g, dob, sig, wdep, "fp64", kw)
    m2, r2 = run_gpu(gj, w, g, dob, sig, wdep, "fp64", kw, graph=graph)
    assert r1["iterations"] == r2["iterations"] == 12
    for i in range(2):
        assert rel(m2[i], m1[i]) <= 1e-12


@pytest.mark.parametrize("npad", [(512, 512), (256, 512), (1024, 32), (1024, 1024)])
def test_joint_fp32_on_the_512_kernels(small, npad):
    """The same solve with 512 x 512 (or 256 x 512) embeddings, served by the
    specialised kernels."""
    gj = lib()
    w, g, A, dob, sig, wdep = small
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(KW))
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, "fp32", KW, npad=npad)
    assert rep["iterations"] == 50
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= 1e-3, (i, rel(m[i], ref.m[i]))
    for k in (0, 1, 10, 49):
        for i in range(2):
            assert rep["history"][k]["phi"][i] == pytest.approx(ref.history[k]["phi"][i], rel=1e-3)


@pytest.mark.parametrize("graph", [False, True])
def test_fast_graph_and_eager_agree(small, graph):
    gj = lib()
    w, g, A, dob, sig, wdep = small
    kw = dict(KW, kmax=10)
    m1, r1 = run_gpu(gj, w, g, dob, sig, wdep, "fp32", kw, npad=(512, 512))
    m2, r2 = run_gpu(gj, w, g, dob, sig, wdep, "fp32", kw, graph=graph, npad=(512, 512))
    for i in range(2):
        # dot products are summed with floating-point atomics: agreement to rounding
        assert rel(m2[i], m1[i]) <= 1e-5


@pytest.mark.parametrize("anchor", ["apriori", "previous"])
@pytest.mark.parametrize("path", ["fp64", "fp32_512", "fp32_256"])
def test_a_priori_model_and_hard_weights(small, path, anchor):
    """m_apr in the Lp factor and the anchor (Eq. WL, RRCG:4) and W_hard in W (Eq. W),
    on the generic FP64 kernels and on the 512 x 512 FP32 kernels."""
    gj = lib()
    w, g, A, dob, sig, wdep = small
    m_apr = [synth.smooth_blocky(g, 0.3, seed=21), synth.smooth_blocky(g, 0.03, seed=22)]
    w_hard = [synth.uniform_model(g, 0.5, 2.0, seed=23), synth.uniform_model(g, 0.5, 2.0, seed=24)]
    kw = dict(KW, kmax=20, anchor=anchor)
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(kw), m_apr=m_apr, w_hard=w_hard)
    prec, npad, tol = {"fp64": ("fp64", (0, 0), 1e-8), "fp32_512": ("fp32", (512, 512), 1e-3),
                       "fp32_256": ("fp32", (256, 512), 1e-3)}[path]
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, prec, kw, npad=npad, m_apr=m_apr, w_hard=w_hard)
    assert rep["iterations"] == 20
    if prec == "fp64":
        compare_history(rep["history"], ref.history, tol)
    for k in (0, 1, 10, 19):
        for i in range(2):
            assert rep["history"][k]["phi"][i] == pytest.approx(ref.history[k]["phi"][i], rel=tol), (k, i)
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= tol, (i, rel(m[i], ref.m[i]))


@pytest.fixture(scope="module")
def ragged():
    w = synth.ragged_joint()
    return (w,) + joint_case(w)


@pytest.mark.parametrize("npad", [(512, 512), (256, 512), (1024, 30), (1024, 1024)])
@pytest.mark.parametrize("optional", [False, True])
def test_fast_solver_partial_line_groups(ragged, optional, npad):
    """13 rows per layer: the 512 kernels' cell-line passes, which take aligned groups
    of four rows, end every layer with a one-row group.  With and without hard
    weights, which select the kernels that read the optional rows.  (An a-priori
    model is left out here: near m = m_apr the L1 factor of Eq. WL is steep enough to
    amplify FP32 rounding of m - m_apr, so FP32 solves with one drift from the FP64
    oracle by up to 1e-2 in 20 iterations on this grid, on the generic kernels as
    well as these; FP64 keeps 1e-11.  The a-priori model is covered by
    test_a_priori_model_and_hard_weights.)"""
    gj = lib()
    w, g, A, dob, sig, wdep = ragged
    probe = gj.bttb_setup(g, "gravity", precision="fp32", npad=npad)
    assert probe.info.fast_path == (2 if npad[0] == 1024 else 1)
    probe.close()
    kw = dict(KW, kmax=20)
    extra = {}
    if optional:
        extra = dict(w_hard=[synth.uniform_model(g, 0.5, 2.0, seed=33), synth.uniform_model(g, 0.5, 2.0, seed=34)])
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(kw), **extra)
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, "fp32", kw, npad=npad, **extra)
    assert rep["iterations"] == 20
    for k in range(20):
        for i in range(2):
            assert rep["history"][k]["phi"][i] == pytest.approx(ref.history[k]["phi"][i], rel=1e-4), (k, i)
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= 1e-4, (i, rel(m[i], ref.m[i]))


@pytest.fixture(scope="module")
def odd():
    w = synth.odd_joint()
    return (w,) + joint_case(w)


@pytest.mark.parametrize("graph", [None, True])
def test_fast256_solver_odd_layers(odd, graph):
    """20x11x7 on the 256-row kernels: seven layers make the last layer pair of every
    column half empty; Phi every iteration and the models against the FP64 oracle,
    eager and graph-replayed."""
    gj = lib()
    w, g, A, dob, sig, wdep = odd
    probe = gj.bttb_setup(g, "gravity", precision="fp32", npad=(256, 512))
    assert probe.info.fast_path == 1
    probe.close()
    kw = dict(KW, kmax=20)
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(kw))
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, "fp32", kw, npad=(256, 512), graph=graph)
    assert rep["iterations"] == 20
    for k in range(20):
        for i in range(2):
            assert rep["history"][k]["phi"][i] == pytest.approx(ref.history[k]["phi"][i], rel=1e-4), (k, i)
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= 1e-4, (i, rel(m[i], ref.m[i]))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_buffer_solve_matches_oracle(small, prec):
    """gj_rrcg_joint_solve_host: numpy inputs, the library copies in and out."""
    gj = lib()
    w, g, A, dob, sig, wdep = small
    kw = dict(KW, kmax=15)
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(kw))
    npad = (0, 0) if prec == "fp64" else (512, 512)
    ops = [gj.bttb_setup(g, "gravity", precision=prec, npad=npad),
           gj.bttb_setup(g, "magnetic", w.mag, precision=prec, npad=npad)]
    nd = np.float64 if prec == "fp64" else np.float32
    host = lambda xs: [np.ascontiguousarray(x, dtype=nd) for x in xs]
    m = host([np.zeros(g.n), np.zeros(g.n)])
    rep = gj.rrcg_joint_solve_host(ops, gj.solver_params(**kw), host(dob), host(sig), host(wdep), m)
    assert rep["iterations"] == 15 and rep["status"] == 0
    assert rep["h2d_bytes"] == (2 * (2 * g.s + g.nz + g.n)) * nd().itemsize
    tol = 1e-9 if prec == "fp64" else 1e-3
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= tol, (i, rel(m[i], ref.m[i]))


@pytest.mark.parametrize("path", [("fp64", (0, 0)), ("fp32", (512, 512))])
def test_solve_with_padding_prisms_and_non_square_grid(path):
    """Stations a subset of the surface prisms (padding prisms left of and below the
    first station, Sec. 2.7.1), dx != dy, variable layer thickness, one layer group
    of 9 rows: the joint solve against the FP64 oracle on both kernel families."""
    gj = lib()
    prec, npad = path
    g = synth.uniform_grid(11, 9, 14, 13, 5, 40.0, off_x=2, off_y=3)
    g.dy = 55.0
    g.z_edges = np.concatenate([[0.0], np.cumsum(np.linspace(25.0, 70.0, g.nz))])
    mag = synth.Mag(50000.0, 60.0, 10.0)
    A = [oop.dense_matrix(g, oop.GRAVITY), oop.dense_matrix(g, oop.MAGNETIC, mag)]
    mt = [synth.smooth_blocky(g, 0.8, 71, n_boxes=2, sigma=2.0), synth.smooth_blocky(g, 0.08, 72, n_boxes=2, sigma=2.0)]
    e = synth.standard_normal((2, g.s), 73)
    obs = [owt.noisy_data(A[i] @ mt[i], 0.01, 0.01, e[i]) for i in range(2)]
    dob, sig = [o[0] for o in obs], [o[1] for o in obs]
    wdep = [owt.depth_weights(g.z_edges, 2.0), owt.depth_weights(g.z_edges, 3.0)]
    kw = dict(KW, kmax=15)
    ref = run_oracle(g, A, dob, sig, wdep, oracle_params(kw))
    w = synth.Workload("padded", g, mag, tuple(mt), (e[0], e[1]))
    m, rep = run_gpu(gj, w, g, dob, sig, wdep, prec, kw, npad=npad)
    assert rep["iterations"] == 15
    tol = 1e-9 if prec == "fp64" else 1e-4
    for k in range(16):
        for i in range(2):
            assert rep["history"][k]["phi"][i] == pytest.approx(ref.history[k]["phi"][i], rel=tol), (k, i)
    for i in range(2):
        assert rel(m[i], ref.m[i]) <= (1e-9 if prec == "fp64" else 1e-3), (i, rel(m[i], ref.m[i]))
