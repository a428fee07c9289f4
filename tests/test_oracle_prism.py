"""Pins for the closed-form prism fields of the oracle (Sec. 2.1, Haaz and
Rao & Babu forms, not printed in the paper): cubature of the integrands,
Laplace's equation, Poisson's relation, the Bouguer slab, far-field point
sources, symmetries and the air-side limit on a top face."""
import numpy as np
import pytest

from oracle import prism
from tests.quadrature import gl_box

PRISMS = [
    # x1, x2, y1, y2, z1, z2 ; station (x0, y0, z0)
    ((0.0, 100.0, 0.0, 50.0, 10.0, 90.0), (50.0, 25.0, -20.0)),
    ((-30.0, 70.0, 40.0, 140.0, 0.0, 100.0), (0.0, 0.0, -35.0)),
    ((100.0, 200.0, -50.0, 50.0, 200.0, 300.0), (0.0, 0.0, 0.0)),
    ((-75.0, -25.0, -25.0, 25.0, 50.0, 100.0), (0.0, 0.0, -10.0)),
]


def gz_integrand(x0, y0, z0):
    def f(X, Y, Z):
        u, v, w = X - x0, Y - y0, Z - z0
        return w / (u * u + v * v + w * w) ** 1.5
    return f


@pytest.mark.parametrize("box,st", PRISMS)
def test_gravity_matches_cubature(box, st):
    x1, x2, y1, y2, z1, z2 = box
    ref = prism.GRAV_UNIT * gl_box(gz_integrand(*st), x1, x2, y1, y2, z1, z2, pts=20, sub=6)
    got = prism.prism_gz(*st, *box)
    assert got == pytest.approx(ref, rel=1e-9)


def hess_integrand(a, b, x0, y0, z0):
    def f(X, Y, Z):
        d = (X - x0, Y - y0, Z - z0)
        R2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
        return (3.0 * d[a] * d[b] - (R2 if a == b else 0.0)) / R2 ** 2.5
    return f


@pytest.mark.parametrize("box,st", PRISMS)
def test_hessian_matches_cubature(box, st):
    x1, x2, y1, y2, z1, z2 = box
    got = prism.prism_hessian(*st, *box)
    names = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    scale = max(abs(g) for g in got)
    for (a, b), g in zip(names, got):
        ref = gl_box(hess_integrand(a, b, *st), x1, x2, y1, y2, z1, z2, pts=20, sub=6)
        assert abs(g - ref) <= 1e-8 * scale, (a, b, g, ref)


def test_laplace_trace_vanishes_including_top_face():
    rng = np.random.default_rng(0)
    for _ in range(50):
        x1, y1 = rng.uniform(-200, 200, 2)
        wx, wy, wz = rng.uniform(10, 150, 3)
        z1 = rng.choice([0.0, rng.uniform(0, 100)])
        x0 = (np.floor(x1 / 10) + 0.5) * 10 if rng.random() < 0.5 else rng.uniform(-300, 300)
        h = prism.prism_hessian(x0 + 0.37, rng.uniform(-300, 300), 0.0, x1, x1 + wx, y1, y1 + wy, z1, z1 + wz)
        tr = h[0] + h[1] + h[2]
        assert abs(tr) <= 1e-12 * max(1.0, max(abs(t) for t in h[:3]))


def test_poisson_relation_hzz_is_depth_derivative_of_gz():
    box = (-40.0, 60.0, -30.0, 50.0, 20.0, 120.0)
    st = (5.0, -7.0, -15.0)
    h = 1e-3
    up = prism.prism_gz(st[0], st[1], st[2] + h, *box) / prism.GRAV_UNIT
    dn = prism.prism_gz(st[0], st[1], st[2] - h, *box) / prism.GRAV_UNIT
    fd = (up - dn) / (2 * h)
    hzz = prism.prism_hessian(*st, *box)[2]
    assert fd == pytest.approx(hzz, rel=1e-6)


def test_bouguer_slab_limit():
    # a wide thin prism under the station tends to 2 pi G rho t (textbook slab)
    # (the finite plate misses a solid-angle fraction of about z / (pi L / 2 sqrt 2))
    t = 50.0
    L = 1.0e8
    g = prism.prism_gz(0.0, 0.0, 0.0, -L, L, -L, L, 100.0, 100.0 + t)
    slab = 2.0 * np.pi * prism.GRAV_UNIT * t
    assert g == pytest.approx(slab, rel=1e-5)


def test_far_field_point_mass_and_dipole():
    a = 10.0
    box = (-a / 2, a / 2, -a / 2, a / 2, 1000.0 - a / 2, 1000.0 + a / 2)
    V = a ** 3
    st = (300.0, -200.0, 0.0)
    d = np.array([0.0 - st[0], 0.0 - st[1], 1000.0 - st[2]])
    R = np.linalg.norm(d)
    g = prism.prism_gz(*st, *box)
    assert g == pytest.approx(prism.GRAV_UNIT * V * d[2] / R ** 3, rel=1e-4)
    H = prism.prism_hessian(*st, *box)
    full = np.array([[H[0], H[3], H[4]], [H[3], H[1], H[5]], [H[4], H[5], H[2]]])
    ref = V * (3.0 * np.outer(d, d) - R * R * np.eye(3)) / R ** 5
    assert np.allclose(full, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())


def test_top_face_is_the_air_side_limit():
    box = (-25.0, 25.0, -25.0, 25.0, 0.0, 50.0)
    on = prism.prism_gz(0.0, 0.0, 0.0, *box)
    for d in (1e-3, 1e-5, 1e-7):
        above = prism.prism_gz(0.0, 0.0, -d, *box)
        assert abs(above - on) <= 2e-3 * d / 1e-3 * abs(on) + 1e-12
    hon = prism.prism_hessian(0.0, 0.0, 0.0, *box)
    habove = prism.prism_hessian(0.0, 0.0, -1e-7, *box)
    assert np.allclose(hon, habove, atol=1e-5)


def test_vertical_inclination_reduces_to_hzz():
    box = (10.0, 60.0, -20.0, 30.0, 0.0, 40.0)
    st = (0.0, 0.0, 0.0)
    dT = prism.prism_dT(*st, *box, 50000.0, 90.0, 0.0)
    assert dT == pytest.approx(50000.0 / (4 * np.pi) * prism.prism_hessian(*st, *box)[2], rel=1e-12)
    t = prism.inducing_direction(60.0, 10.0)
    assert np.linalg.norm(t) == pytest.approx(1.0)
    assert t[2] > 0 and t[1] > t[0] > 0  # down, mostly north, a little east


# ---------------------------------------------------------------------------
# Far-field cubature (used for prisms at least FAR sizes from the station, where
# the corner sums cancel)

def _box(off, h=100.0, dz=100.0):
    ox, oy, oz = off
    return ((ox - 0.5) * h, (ox + 0.5) * h, (oy - 0.5) * h, (oy + 0.5) * h, (oz - 0.5) * dz, (oz + 0.5) * dz)


@pytest.mark.parametrize("off", [(8.0, 0.0, 1.5), (5.0, 6.0, 2.5), (6.0, 6.0, 4.0), (1.5, 2.5, 9.0)])
def test_cubature_equals_closed_form_where_both_hold(off):
    """8-12 sizes out the corner sums still keep about 11 digits: both evaluations of
    the Sec. 2.1 integrals agree to 1e-10."""
    x1, x2, y1, y2, z1, z2 = _box(off)
    g_c = prism.prism_gz(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2)
    g_q = prism.prism_gz_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2)
    assert g_q == pytest.approx(g_c, rel=1e-10)
    m_c = prism.prism_dT(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, 50000.0, 60.0, 10.0)
    m_q = prism.prism_dT_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, 50000.0, 60.0, 10.0)
    assert m_q == pytest.approx(m_c, rel=1e-10)


@pytest.mark.parametrize("off", [(20.0, 7.0, 3.5), (60.0, 60.0, 30.5), (150.0, 90.0, 12.5)])
def test_cubature_converges_far_out(off):
    x1, x2, y1, y2, z1, z2 = _box(off)
    dist = np.linalg.norm([0.5 * (x1 + x2), 0.5 * (y1 + y2), 0.5 * (z1 + z2)])
    n_rule = int(prism.cubature_order(dist, 100.0))
    for n_lo, n_hi in ((n_rule, 7), (5, 7)):
        a = prism.prism_gz_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, n=n_lo)
        b = prism.prism_gz_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, n=n_hi)
        assert a == pytest.approx(b, rel=2e-13)
        a = prism.prism_dT_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, 5e4, 60.0, 10.0, n=n_lo)
        b = prism.prism_dT_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, 5e4, 60.0, 10.0, n=n_hi)
        assert a == pytest.approx(b, rel=2e-13)
    # and tends to the point mass: G rho V w / R^3 (mGal per g/cc)
    d = np.array([0.5 * (x1 + x2), 0.5 * (y1 + y2), 0.5 * (z1 + z2)])
    R = np.linalg.norm(d)
    pm = prism.GRAV_UNIT * (x2 - x1) * (y2 - y1) * (z2 - z1) * d[2] / R ** 3
    assert prism.prism_gz_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2) == pytest.approx(pm, rel=3.0 / (R / 100.0) ** 2)


def test_cubature_hessian_trace_vanishes():
    """Laplace: the three axis-aligned inducing directions sum to the trace of the
    Hessian of 1/R, zero away from the source."""
    x1, x2, y1, y2, z1, z2 = _box((30.0, 11.0, 6.5))
    s = sum(prism.prism_dT_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, 4 * np.pi, inc, dec)
            for inc, dec in ((0.0, 90.0), (0.0, 0.0), (90.0, 0.0)))
    scale = abs(prism.prism_dT_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, 4 * np.pi, 90.0, 0.0))
    assert abs(s) <= 1e-12 * scale


@pytest.mark.skipif(np.finfo(np.longdouble).nmant < 63, reason="needs extended precision")
def test_cubature_against_extended_precision_corner_sums():
    """Far out the FP64 corner sums lose digits (the eight terms are ~1e6 times the
    field); in extended precision they keep about 12, and the cubature matches them."""
    L = np.longdouble

    def gz_ld(x1, x2, y1, y2, z1, z2):
        def f(u, v, w):
            u, v, w = L(u), L(v), L(w)
            R = np.sqrt(u * u + v * v + w * w)
            lg = lambda a, b, c: np.log(a + R) if a >= 0 else np.log((b * b + c * c) / (R - a))
            return -(u * lg(v, u, w) + v * lg(u, v, w) - w * np.arctan2(u * v, w * R))
        s = L(0)
        for i, u in ((1, x1), (2, x2)):
            for j, v in ((1, y1), (2, y2)):
                for k, w in ((1, z1), (2, z2)):
                    s += (-1) ** (i + j + k) * f(u, v, w)
        return float(s * L(prism.GRAV_UNIT))

    for off in [(40.0, 40.0, 20.5), (24.0, 3.0, 10.5)]:
        x1, x2, y1, y2, z1, z2 = _box(off)
        ref = gz_ld(x1, x2, y1, y2, z1, z2)
        assert prism.prism_gz_cubature(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2) == pytest.approx(ref, rel=1e-11)


def test_cubature_with_an_offset_lifted_station():
    """The cubature measures the prism from the station: moving both together changes
    nothing, and with a station above the mesh (z0 < 0) it still equals the closed
    form 8-12 sizes out."""
    x1, x2, y1, y2, z1, z2 = _box((7.0, 5.0, 4.5))
    x0, y0, z0 = 321.0, -47.0, -15.0
    for fun, extra in ((prism.prism_gz_cubature, ()), (prism.prism_dT_cubature, (5e4, 60.0, 10.0))):
        a = fun(0.0, 0.0, 0.0, x1, x2, y1, y2, z1, z2, *extra)
        b = fun(x0, y0, z0, x1 + x0, x2 + x0, y1 + y0, y2 + y0, z1 + z0, z2 + z0, *extra)
        assert b == pytest.approx(a, rel=1e-13)
    g_c = prism.prism_gz(x0, y0, z0, x1, x2, y1, y2, z1, z2)
    g_q = prism.prism_gz_cubature(x0, y0, z0, x1, x2, y1, y2, z1, z2)
    assert g_q == pytest.approx(g_c, rel=1e-10)
    m_c = prism.prism_dT(x0, y0, z0, x1, x2, y1, y2, z1, z2, 5e4, 60.0, 10.0)
    m_q = prism.prism_dT_cubature(x0, y0, z0, x1, x2, y1, y2, z1, z2, 5e4, 60.0, 10.0)
    assert m_q == pytest.approx(m_c, rel=1e-10)
