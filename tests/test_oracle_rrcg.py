"""Pins for the oracle's RRCG joint solve (Eq. RRCG:1-8, Secs. 2.5, 2.6, 2.8).

The nonlinear solve has no closed form; the pins are the special cases that the
mathematics fixes: with lambda = 0, p = 2 and a fixed alpha the iteration is
linear CG on the weighted normal equations (it must decrease the objective
monotonically and reach the direct solve), plus the discrete rules: bounds,
the alpha schedule and its freeze, and the chi^2 stop."""
import numpy as np
import pytest

import synth
from oracle import operator as op
from oracle import weights as wt
from oracle.rrcg import RRCGParams, rrcg_joint


def small_problem(seed=0, nx=6, ny=5, nz=3):
    g = synth.uniform_grid(nx, ny, nx, ny, nz, 50.0)
    mag = synth.Mag(50000.0, 60.0, 10.0)
    A = [op.dense_matrix(g, op.GRAVITY), op.dense_matrix(g, op.MAGNETIC, mag)]
    rng = np.random.default_rng(seed)
    mt = [rng.uniform(0, 1, g.n), rng.uniform(0, 0.1, g.n)]
    d = [A[i] @ mt[i] for i in range(2)]
    sig = [wt.noise_sigma(d[i], 0.01, 0.01) for i in range(2)]
    dobs = [d[i] + sig[i] * rng.standard_normal(g.s) for i in range(2)]
    return g, A, mt, dobs, sig


@pytest.mark.parametrize("scalars", ["joint", "per_field"])
def test_linear_case_is_cg_and_reaches_direct_solve(scalars):
    g, A, mt, dobs, sig = small_problem()
    wdep = [wt.depth_weight_cells(g.z_edges, 2.0, g.nx, g.ny), wt.depth_weight_cells(g.z_edges, 3.0, g.nx, g.ny)]
    alpha = (5.0, 0.02)
    P = RRCGParams(p=(2, 2), alpha1=alpha, q=(1.0, 1.0), lam=(0.0, 0.0), lo=(-1e30, -1e30),
                   hi=(1e30, 1e30), kmax=400, stop_on_chi2=False, scalars=scalars)
    res = rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)],
                     [lambda y, i=i: A[i].T @ y for i in range(2)],
                     dobs, sig, [np.zeros(g.n)] * 2, wdep, P)
    for i in range(2):
        At = (A[i] / sig[i][:, None]) / wdep[i][None, :]
        dt = dobs[i] / sig[i]
        H = At.T @ At + alpha[i] * np.eye(g.n)
        mt_star = np.linalg.solve(H, At.T @ dt)
        m_star = mt_star / wdep[i]
        assert np.linalg.norm(res.m[i] - m_star) <= 1e-8 * np.linalg.norm(m_star)
    P2 = RRCGParams(**{**P.__dict__, "kmax": 1})
    # monotone decrease along one run: recompute the objective at each iterate
    ms = [np.zeros(g.n)] * 2
    prev = np.inf
    for k in range(1, 30):
        r = rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)],
                       [lambda y, i=i: A[i].T @ y for i in range(2)],
                       dobs, sig, ms, wdep, RRCGParams(**{**P2.__dict__, "kmax": k}))
        val = sum(np.sum(((A[i] @ r.m[i] - dobs[i]) / sig[i]) ** 2) + alpha[i] * np.sum((wdep[i] * r.m[i]) ** 2)
                  for i in range(2))
        assert val <= prev * (1 + 1e-12)
        prev = val


def test_bounds_alpha_schedule_and_chi2_stop():
    g, A, mt, dobs, sig = small_problem(seed=5)
    ones = [np.ones(g.n), np.ones(g.n)]
    P = RRCGParams(p=(1, 1), alpha1=(100.0, 100.0), q=(0.8, 0.9), alpha_min=(1.0, 5.0),
                   lam=(10.0, 200.0), lo=(0.0, 0.0), hi=(1.0, 0.1), kmax=60, stop_on_chi2=True)
    res = rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)],
                     [lambda y, i=i: A[i].T @ y for i in range(2)],
                     dobs, sig, [np.zeros(g.n)] * 2, ones, P)
    for i in range(2):
        assert res.m[i].min() >= P.lo[i] and res.m[i].max() <= P.hi[i]
    target = g.s + np.sqrt(2 * g.s)
    hist = res.history
    for i in range(2):
        a_prev = P.alpha1[i]
        frozen = False
        for k, rec in enumerate(hist):
            if rec["phi"][i] <= target:
                frozen = True
            if k > 0:
                want = a_prev if frozen else max(P.q[i] * a_prev, P.alpha_min[i])
                assert rec["alpha"][i] == pytest.approx(want, rel=1e-15)
            a_prev = rec["alpha"][i]
    if res.converged:
        assert all(hist[-1]["satisfied"]) and res.iterations < P.kmax
    else:
        assert res.iterations == P.kmax


def test_first_iterate_weights_and_first_direction():
    # c14: m0 = m_apr = 0 gives W_L = eps^(-1/2) everywhere, l_G = 0, p_0 = l_0
    g, A, mt, dobs, sig = small_problem(seed=9)
    eps2 = 1e-9
    w = wt.lp_weight(np.zeros(5), np.zeros(5), eps2, 1)
    assert np.allclose(w, eps2 ** -0.25)
    P = RRCGParams(p=(1, 1), eps2=eps2, alpha1=(10.0, 10.0), q=(1, 1), lam=(5.0, 5.0),
                   lo=(-1e30, -1e30), hi=(1e30, 1e30), kmax=1, stop_on_chi2=False, scalars="joint")
    res = rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)],
                     [lambda y, i=i: A[i].T @ y for i in range(2)],
                     dobs, sig, [np.zeros(g.n)] * 2, [np.ones(g.n)] * 2, P)
    # one step from zero: m1 = -s W^-1 l_0 with l_0 = W^-1 A^T W_d^2 (-d)
    Wl = eps2 ** -0.25
    l0 = [(A[i].T @ (-dobs[i] / sig[i] ** 2)) / Wl for i in range(2)]
    q = [(A[i] @ (l0[i] / Wl)) / sig[i] for i in range(2)]
    s = sum(l0[i] @ l0[i] for i in range(2)) / sum(q[i] @ q[i] + 15.0 * (l0[i] @ l0[i]) for i in range(2))
    for i in range(2):
        assert np.allclose(res.m[i], -s * l0[i] / Wl, rtol=1e-12, atol=1e-14)
