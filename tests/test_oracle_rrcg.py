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


# ---------------------------------------------------------------------------
# Pins of the Gramian coupling (RRCG:2-4), the weighted-space branch (Eq.
# steepestascenta/b, Appendix A) and the previous-model anchor (RRCG:4 as
# printed).  Each compares a direction the oracle takes with half the gradient
# of an objective written out below from Eq. (GlobalFunction1) / (GlobalFunction2)
# and differentiated numerically, so that no line of the oracle is reused.

def written_out_objective(A, dobs, sig, m1, m2, alpha, lam, w=(1.0, 1.0), anchor=(0.0, 0.0)):
    """Eq. (GlobalFunction1) with one Lagrange weight: data misfit ||W_d (A m - d)||^2,
    stabiliser alpha ||w (m - anchor)||^2 and lam * det [[m1.m1, m1.m2], [m2.m1, m2.m2]]."""
    tot = 0.0
    for i, m in enumerate((m1, m2)):
        r = (A[i] @ m - dobs[i]) / sig[i]
        tot += float(r @ r) + alpha[i] * float(np.sum((w[i] * (m - anchor[i])) ** 2))
    gram = np.array([[m1 @ m1, m1 @ m2], [m2 @ m1, m2 @ m2]])
    return tot + lam * float(np.linalg.det(gram))


def half_gradient(fun, x1, x2, h=1e-5):
    """(1/2) grad of fun(x1, x2) by central differences, one coordinate at a time."""
    out = []
    for which in range(2):
        base = (x1, x2)[which]
        g = np.empty_like(base)
        for j in range(base.size):
            e = np.zeros_like(base)
            e[j] = h
            if which == 0:
                g[j] = (fun(x1 + e, x2) - fun(x1 - e, x2)) / (2 * h)
            else:
                g[j] = (fun(x1, x2 + e) - fun(x1, x2 - e)) / (2 * h)
        out.append(0.5 * g)
    return out


def one_step(A, dobs, sig, m0, w_static, P, m_apr=None):
    return rrcg_joint([lambda x, i=i: A[i] @ x for i in range(2)],
                      [lambda y, i=i: A[i].T @ y for i in range(2)],
                      dobs, sig, m0, w_static, P, m_apr=m_apr)


FREE = dict(lo=(-1e30, -1e30), hi=(1e30, 1e30), stop_on_chi2=False, q=(1.0, 1.0))


def nonzero_start(g, seed):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.1, 1.0, g.n), rng.uniform(0.01, 0.1, g.n)]


@pytest.mark.parametrize("lam", [(3000.0, 3000.0), (2000.0, 6000.0)])
def test_first_direction_is_half_gradient_with_gramian(lam):
    """W = I (p = 2, unit static weights): l_0 of RRCG:4 from a nonzero m_0 equals half
    the gradient of P = misfit + alpha ||m||^2 + lambda_i S_G, field by field (with
    lambda_1 != lambda_2, field i's direction is the gradient of the objective that
    carries lambda_i).  The lambda l_G share is nonzero here, unlike from m_0 = 0."""
    g, A, mt, dobs, sig = small_problem(seed=11)
    m0 = nonzero_start(g, 12)
    alpha = (3.0, 0.4)
    P = RRCGParams(p=(2, 2), alpha1=alpha, lam=lam, kmax=1, scalars="joint", **FREE)
    res = one_step(A, dobs, sig, m0, [np.ones(g.n)] * 2, P)
    s = res.history[0]["s"]
    l0 = [(m0[i] - res.m[i]) / s[i] for i in range(2)]
    for i in range(2):
        f = lambda x1, x2: written_out_objective(A, dobs, sig, x1, x2, alpha, lam[i])
        want = half_gradient(f, m0[0], m0[1])[i]
        assert np.linalg.norm(l0[i] - want) <= 1e-7 * np.linalg.norm(want), i
        assert res.history[0]["ll"][i] == pytest.approx(float(l0[i] @ l0[i]), rel=1e-12)
    # the Gramian share is a sizeable part of each direction (the pin would see it vanish)
    sg = lambda x1, x2: float(np.linalg.det(np.array([[x1 @ x1, x1 @ x2], [x2 @ x1, x2 @ x2]])))
    hg = half_gradient(sg, m0[0], m0[1], h=1e-6)
    for i in range(2):
        assert lam[i] * np.linalg.norm(hg[i]) > 0.2 * np.linalg.norm(l0[i]), i


def test_gramian_term_with_l1_weights_is_unweighted_half_gradient():
    """p = 1 with a non-uniform W_L from a nonzero m_0: the RRCG:2-4 Gramian share of
    l_0 is lambda_i times half the gradient of S_G in the ORIGINAL model space (no W^-1,
    no factor 2).  The share is isolated as the difference of the directions with and
    without lambda; l_0 = W (m_0 - m_1) / s for the frozen W_0."""
    g, A, mt, dobs, sig = small_problem(seed=13)
    m0 = nonzero_start(g, 14)
    wdep = [wt.depth_weight_cells(g.z_edges, 2.0, g.nx, g.ny), wt.depth_weight_cells(g.z_edges, 3.0, g.nx, g.ny)]
    lam = (7.0, 90.0)
    W0 = [wdep[i] * wt.lp_weight(m0[i], 0.0, 1e-9, 1) for i in range(2)]
    dirs = {}
    for key, lm in (("on", lam), ("off", (0.0, 0.0))):
        P = RRCGParams(p=(1, 1), alpha1=(2.0, 5.0), lam=lm, kmax=1, scalars="joint", **FREE)
        res = one_step(A, dobs, sig, m0, wdep, P)
        s = res.history[0]["s"]
        dirs[key] = [W0[i] * (m0[i] - res.m[i]) / s[i] for i in range(2)]
    sg = lambda x1, x2: float(np.linalg.det(np.array([[x1 @ x1, x1 @ x2], [x2 @ x1, x2 @ x2]])))
    hg = half_gradient(sg, m0[0], m0[1], h=1e-6)
    for i in range(2):
        share = dirs["on"][i] - dirs["off"][i]
        want = lam[i] * hg[i]
        assert np.linalg.norm(share - want) <= 1e-6 * np.linalg.norm(want), i


def test_l1_weight_squares_to_the_l1_norm():
    """Eq. WL is the IRLS form of the L1 stabiliser: sum (W_L (m - m_apr))^2 =
    sum d^2 / sqrt(d^2 + eps^2) tends to ||m - m_apr||_1 as eps -> 0."""
    rng = np.random.default_rng(15)
    m = rng.uniform(-1, 1, 500)
    ma = rng.uniform(-0.5, 0.5, 500)
    d = m - ma
    for eps2 in (1e-9, 1e-12):
        val = np.sum((wt.lp_weight(m, ma, eps2, 1) * d) ** 2)
        assert val == pytest.approx(np.sum(np.abs(d)), rel=10 * eps2 / np.min(d * d))
    # p = 2 is the identity (minimum-length variant, Sec. 3.1.5)
    assert np.all(wt.lp_weight(m, ma, 1e-9, 2) == 1.0)


def test_monotone_decrease_with_equal_lambdas_and_frozen_weights():
    """Sec. 8(c-iii) reading: lambda_1 = lambda_2, W frozen (p = 2, unit weights), fixed
    alpha and a small lambda: every iterate lowers the written-out objective."""
    g, A, mt, dobs, sig = small_problem(seed=16)
    m0 = nonzero_start(g, 17)
    alpha, lam = (2.0, 0.5), 0.5
    prev = written_out_objective(A, dobs, sig, m0[0], m0[1], alpha, lam)
    for k in range(1, 26):
        P = RRCGParams(p=(2, 2), alpha1=alpha, lam=(lam, lam), kmax=k, scalars="joint", **FREE)
        res = one_step(A, dobs, sig, m0, [np.ones(g.n)] * 2, P)
        val = written_out_objective(A, dobs, sig, res.m[0], res.m[1], alpha, lam)
        assert val <= prev * (1 + 1e-13), k
        prev = val


def test_weighted_space_gramian_branch():
    """Eq. steepestascenta/b with scalar weights W_i = w_i I (p = 2): the first direction
    is half the gradient, with respect to m~ = W m, of the weighted objective
    ||W_d (A m~/w - d)||^2 + alpha ||m~||^2 + lambda S_G(m~_1, m~_2) (Eq. GlobalFunction2),
    and the reported weighted Gramian is (w_1 w_2)^2 S_G (Appendix A)."""
    g, A, mt, dobs, sig = small_problem(seed=18)
    m0 = nonzero_start(g, 19)
    w = (1.7, 0.6)
    alpha, lam = (1.5, 0.8), 0.02
    P = RRCGParams(p=(2, 2), alpha1=alpha, lam=(lam, lam), kmax=1, scalars="joint", gramian_space="weighted",
                   **FREE)
    res = one_step(A, dobs, sig, m0, [np.full(g.n, w[0]), np.full(g.n, w[1])], P)
    s = res.history[0]["s"]
    l0 = [w[i] * (m0[i] - res.m[i]) / s[i] for i in range(2)]

    def weighted(t1, t2):
        tot = 0.0
        for i, t in enumerate((t1, t2)):
            r = (A[i] @ (t / w[i]) - dobs[i]) / sig[i]
            tot += float(r @ r) + alpha[i] * float(t @ t)
        return tot + lam * float(np.linalg.det(np.array([[t1 @ t1, t1 @ t2], [t2 @ t1, t2 @ t2]])))

    mt0 = [w[i] * m0[i] for i in range(2)]
    want = half_gradient(weighted, mt0[0], mt0[1])
    for i in range(2):
        assert np.linalg.norm(l0[i] - want[i]) <= 1e-7 * np.linalg.norm(want[i]), i
    h0 = res.history[0]
    assert h0["S_G_space"] == pytest.approx((w[0] * w[1]) ** 2 * h0["S_G"], rel=1e-12)
    # the original-space branch reports S_G itself
    P2 = RRCGParams(**{**P.__dict__, "gramian_space": "original"})
    res2 = one_step(A, dobs, sig, m0, [np.full(g.n, w[0]), np.full(g.n, w[1])], P2)
    assert res2.history[0]["S_G_space"] == res2.history[0]["S_G"]


@pytest.mark.parametrize("anchor", ["apriori", "previous"])
def test_second_direction_and_regulariser_anchor(anchor):
    """k = 1 from m_0 != 0, W = I: l_1 = p_1 - beta_1 p_0 must equal half the gradient at
    m_1 of the objective whose stabiliser is alpha ||m - a||^2 with a = m_apr (= 0,
    Eq. FirstVariation) or a = m_0 (the previous model, RRCG:4 as printed); beta_1 is
    ||l_1||^2 / ||l_0||^2 over both fields (RRCG:5, joint scalars)."""
    g, A, mt, dobs, sig = small_problem(seed=20)
    m0 = nonzero_start(g, 21)
    alpha, lam = (4.0, 1.0), 0.3
    ones = [np.ones(g.n)] * 2
    P1 = RRCGParams(p=(2, 2), alpha1=alpha, lam=(lam, lam), kmax=1, scalars="joint", anchor=anchor, **FREE)
    P2 = RRCGParams(**{**P1.__dict__, "kmax": 2})
    r1 = one_step(A, dobs, sig, m0, ones, P1)
    r2 = one_step(A, dobs, sig, m0, ones, P2)
    m1, m2 = r1.m, r2.m
    s0, s1 = r2.history[0]["s"], r2.history[1]["s"]
    beta1 = r2.history[1]["beta"]
    p0 = [(m0[i] - m1[i]) / s0[i] for i in range(2)]
    p1 = [(m1[i] - m2[i]) / s1[i] for i in range(2)]
    l1 = [p1[i] - beta1[i] * p0[i] for i in range(2)]
    a = (m0[0], m0[1]) if anchor == "previous" else (0.0, 0.0)
    f = lambda x1, x2: written_out_objective(A, dobs, sig, x1, x2, alpha, lam, anchor=a)
    want = half_gradient(f, m1[0], m1[1])
    for i in range(2):
        assert np.linalg.norm(l1[i] - want[i]) <= 1e-6 * np.linalg.norm(want[i]), i
    f0 = lambda x1, x2: written_out_objective(A, dobs, sig, x1, x2, alpha, lam)
    l0 = half_gradient(f0, m0[0], m0[1])
    b = sum(float(x @ x) for x in want) / sum(float(x @ x) for x in l0)
    assert beta1[0] == beta1[1] == pytest.approx(b, rel=1e-6)


def test_depth_weights_closed_form():
    """Reading of the depth weighting (Li & Oldenburg form at layer centres): uniform
    layers of thickness dz from the surface have centres (k + 1/2) dz, so layer k gets
    (2k + 1)^(-beta/2); the top layer has weight 1 and deeper ones decrease."""
    z = np.arange(11) * 37.5
    for beta in (2.0, 3.0):
        w = wt.depth_weights(z, beta)
        np.testing.assert_allclose(w, (2.0 * np.arange(10) + 1.0) ** (-beta / 2.0), rtol=1e-15)
        assert w[0] == 1.0 and np.all(np.diff(w) < 0)
    cells = wt.depth_weight_cells(z, 2.0, 3, 2)
    assert cells.shape == (60,) and np.all(cells[:6] == 1.0) and np.all(cells[6:12] == cells[6])
