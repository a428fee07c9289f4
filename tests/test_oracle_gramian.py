"""Pins for the oracle's Gramian (Eq. Gramian, RRCG:2-3, Appendix A)."""
import numpy as np
import pytest

from oracle import gramian as gm


def test_lagrange_identity_brute_force():
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 64):
        a = rng.standard_normal(n)
        b = rng.standard_normal(n)
        brute = 0.5 * sum((a[j] * b[k] - a[k] * b[j]) ** 2 for j in range(n) for k in range(n))
        assert gm.gramian(a, b) == pytest.approx(brute, rel=1e-12, abs=1e-12)


def test_collinear_models_give_zero_and_value_is_nonnegative():
    rng = np.random.default_rng(1)
    a = rng.uniform(0, 1, 500)
    assert abs(gm.gramian(a, 0.1 * a)) <= 1e-12 * (a @ a) ** 2 * 0.01
    for _ in range(20):
        b = rng.standard_normal(500)
        assert gm.gramian(a, b) >= 0
    # orthogonal unit vectors: determinant 1
    e1 = np.zeros(4); e1[0] = 1
    e2 = np.zeros(4); e2[2] = 1
    assert gm.gramian(e1, e2) == 1.0


def test_scalar_weights_scale_by_product_squared():
    # Appendix A: W_i = w_i I gives S~_G = (w1 w2)^2 S_G
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal(50), rng.standard_normal(50)
    w1, w2 = 3.0, 0.25
    assert gm.gramian(w1 * a, w2 * b) == pytest.approx((w1 * w2) ** 2 * gm.gramian(a, b), rel=1e-12)


def test_ascent_directions_are_half_gradients():
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal(30), rng.standard_normal(30)
    l1, l2 = gm.ascent_directions(a, b)
    h = 1e-6
    for j in range(30):
        e = np.zeros(30); e[j] = h
        g1 = (gm.gramian(a + e, b) - gm.gramian(a - e, b)) / (2 * h)
        g2 = (gm.gramian(a, b + e) - gm.gramian(a, b - e)) / (2 * h)
        assert g1 == pytest.approx(2 * l1[j], rel=1e-6, abs=1e-6)
        assert g2 == pytest.approx(2 * l2[j], rel=1e-6, abs=1e-6)
    # the directions vanish for collinear models
    z1, z2 = gm.ascent_directions(a, -2.0 * a)
    assert np.abs(z1).max() <= 1e-12 * (a @ a) * np.abs(a).max() * 4
    assert np.abs(z2).max() <= 1e-12 * (a @ a) * np.abs(a).max() * 4


def test_unweighted_gramian_gradient_in_weighted_variables():
    # Eq. descentrelaS: grad over m~ of S_G(W^-1 m~) = 2 W^-1 l_G
    rng = np.random.default_rng(4)
    m1, m2 = rng.standard_normal(12), rng.standard_normal(12)
    W1, W2 = rng.uniform(0.5, 2, 12), rng.uniform(0.5, 2, 12)
    mt1 = W1 * m1
    l1, _ = gm.ascent_directions(m1, m2)
    h = 1e-6
    for j in range(12):
        e = np.zeros(12); e[j] = h
        fd = (gm.gramian((mt1 + e) / W1, m2) - gm.gramian((mt1 - e) / W1, m2)) / (2 * h)
        assert fd == pytest.approx(2 * l1[j] / W1[j], rel=1e-6, abs=1e-7)
