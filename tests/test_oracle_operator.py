"""Pins for the oracle's sensitivity operators (Eq. d=gm, Sec. 2.7.1):
BTTB structure of each depth block, equality with an independently written
numpy-FFT BCCB product, the adjoint identity, sampled direct sums, symmetries,
and the storage figures the paper prints."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import operator as op

HERE = os.path.dirname(os.path.abspath(__file__))


def small_grids():
    yield synth.uniform_grid(6, 5, 6, 5, 3, 50.0)
    # stations a subset of the surface prisms (padding prisms, Sec. 2.7.1), non-square
    g = synth.uniform_grid(4, 3, 7, 6, 2, 40.0, dz=30.0, off_x=2, off_y=1)
    g.dy = 55.0
    yield g
    yield synth.uniform_grid(5, 7, 5, 7, 4, 25.0)


MAG = synth.Mag(50000.0, 60.0, 10.0)


@pytest.mark.parametrize("field", [op.GRAVITY, op.MAGNETIC])
def test_dense_entries_follow_table(field):
    for g in small_grids():
        A = op.dense_matrix(g, field, MAG)
        K = op.kernel_table(g, field, MAG)
        a0 = g.off_y - (g.ny - 1)
        b0 = g.off_x - (g.nx - 1)
        for j in range(g.s):
            jy, jx = divmod(j, g.sx)
            for c in range(g.n):
                r, rem = divmod(c, g.nx * g.ny)
                iy, ix = divmod(rem, g.nx)
                assert A[j, c] == K[r, jy + g.off_y - iy - a0, jx + g.off_x - ix - b0]


def bccb_forward(K, g, m, Ny, Nx):
    """Independent FFT statement of Sec. 2.7.1: T[c mod N] = K(c + off) for
    c in [-(n-1), s-1]; m in the upper-left corner; keep the upper-left s block."""
    m3 = m.reshape(g.nz, g.ny, g.nx)
    out = np.zeros((g.sy, g.sx))
    for r in range(g.nz):
        T = np.zeros((Ny, Nx))
        for ca in range(-(g.ny - 1), g.sy):
            for cb in range(-(g.nx - 1), g.sx):
                T[ca % Ny, cb % Nx] = K[r, ca + g.ny - 1, cb + g.nx - 1]
        X = np.zeros((Ny, Nx))
        X[:g.ny, :g.nx] = m3[r]
        y = np.fft.ifft2(np.fft.fft2(T) * np.fft.fft2(X)).real
        out += y[:g.sy, :g.sx]
    return out.reshape(-1)


def bccb_adjoint(K, g, rv, Ny, Nx):
    r2 = rv.reshape(g.sy, g.sx)
    out = np.zeros((g.nz, g.ny, g.nx))
    for r in range(g.nz):
        T = np.zeros((Ny, Nx))
        for ca in range(-(g.ny - 1), g.sy):
            for cb in range(-(g.nx - 1), g.sx):
                T[ca % Ny, cb % Nx] = K[r, ca + g.ny - 1, cb + g.nx - 1]
        V = np.zeros((Ny, Nx))
        V[:g.sy, :g.sx] = r2
        y = np.fft.ifft2(np.conj(np.fft.fft2(T)) * np.fft.fft2(V)).real
        out[r] = y[:g.ny, :g.nx]
    return out.reshape(-1)


@pytest.mark.parametrize("field", [op.GRAVITY, op.MAGNETIC])
def test_dense_equals_fft_embedding_for_any_padding(field):
    rng = np.random.default_rng(7)
    for g in small_grids():
        A = op.dense_matrix(g, field, MAG)
        K = op.kernel_table(g, field, MAG)
        m = rng.standard_normal(g.n)
        rv = rng.standard_normal(g.s)
        Nmin_y, Nmin_x = g.sy + g.ny - 1, g.sx + g.nx - 1
        for Ny, Nx in [(Nmin_y, Nmin_x), (Nmin_y + 3, Nmin_x + 1), (16, 16)]:
            f = bccb_forward(K, g, m, Ny, Nx)
            a = bccb_adjoint(K, g, rv, Ny, Nx)
            d = A @ m
            gt = A.T @ rv
            assert np.linalg.norm(f - d) <= 1e-13 * np.linalg.norm(d)
            assert np.linalg.norm(a - gt) <= 1e-13 * np.linalg.norm(gt)


@pytest.mark.parametrize("field", [op.GRAVITY, op.MAGNETIC])
def test_sampled_direct_sums_and_adjoint_identity(field):
    rng = np.random.default_rng(3)
    for g in small_grids():
        A = op.dense_matrix(g, field, MAG)
        K = op.kernel_table(g, field, MAG)
        m = rng.standard_normal(g.n)
        rv = rng.standard_normal(g.s)
        d = op.forward_direct(K, g, m)
        gt = op.adjoint_direct(K, g, rv)
        assert np.allclose(d, A @ m, rtol=1e-13, atol=1e-13 * np.abs(A @ m).max())
        assert np.allclose(gt, A.T @ rv, rtol=1e-13, atol=1e-13 * np.abs(A.T @ rv).max())
        lhs = d @ rv
        rhs = m @ gt
        assert abs(lhs - rhs) <= 1e-13 * (np.abs(d) @ np.abs(rv))


def test_gravity_table_even_and_vertical_magnetic_even():
    g = synth.uniform_grid(6, 6, 6, 6, 3, 50.0)
    K = op.kernel_table(g, op.GRAVITY)
    # corner sums cancel far from the prism: compare against the table's scale
    tol = 1e-12 * np.abs(K).max()
    assert np.allclose(K, K[:, ::-1, :], rtol=0, atol=tol)
    assert np.allclose(K, K[:, :, ::-1], rtol=0, atol=tol)
    Km = op.kernel_table(g, op.MAGNETIC, synth.Mag(50000.0, 90.0, 0.0))
    assert np.allclose(Km, Km[:, ::-1, ::-1], rtol=1e-12, atol=1e-12 * np.abs(Km).max())
    # general inclination: the magnetic block is not symmetric (Sec. 2.7.1)
    Kg = op.kernel_table(g, op.MAGNETIC, synth.Mag(50000.0, 45.0, 45.0))
    assert not np.allclose(Kg, Kg[:, ::-1, ::-1], rtol=1e-6)
    # the magnetic kernel with I = 90 equals (F / 4pi) Hzz: positive right under the station
    assert Km[0, g.ny - 1, g.nx - 1] > 0


def test_storage_figures_printed_in_the_paper():
    gold = json.load(open(os.path.join(HERE, "golden", "storage.json")))
    e = gold["dense_example"]
    assert e["rows"] * e["cols"] * e["bytes_per_real"] / 1e9 == pytest.approx(e["printed_GB"])
    mb = gold["multiple_bodies"]
    g = synth.uniform_grid(mb["sx"], mb["sy"], mb["nx"], mb["ny"], mb["nz"], 100.0)
    a, b = op.table_offsets(g)
    assert [b.size, a.size, g.nz] == mb["printed_transform_shape"]
    dense = 2 * g.s * g.n * 8
    assert dense >= mb["printed_dense_bytes"]
    trans = 2 * a.size * b.size * g.nz * 16
    assert trans / 1e6 == pytest.approx(mb["printed_transform_MB"], rel=0.01)
    assert dense / trans == pytest.approx(mb["printed_reduction"], rel=0.01)


@pytest.mark.parametrize("field", [op.GRAVITY, op.MAGNETIC])
def test_bccb_products_and_dense_from_table_equal_the_dense_product(field):
    """The oracle's FFT evaluation (Sec. 2.7.1) against the plain dense product, for
    the minimal padding, a larger odd padding and a power of two; and the matrix
    assembled from the table against the one assembled from the prisms."""
    rng = np.random.default_rng(17)
    for g in small_grids():
        A = op.dense_matrix(g, field, MAG)
        K = op.kernel_table(g, field, MAG)
        assert np.array_equal(op.dense_from_table(K, g), A)
        m = rng.standard_normal(g.n)
        rv = rng.standard_normal(g.s)
        Nmin_y, Nmin_x = g.sy + g.ny - 1, g.sx + g.nx - 1
        for Ny, Nx in [(Nmin_y, Nmin_x), (Nmin_y + 3, Nmin_x + 1), (16, 16)]:
            B = op.BCCB(K, g, Ny, Nx)
            d, gt = A @ m, A.T @ rv
            assert np.linalg.norm(B.forward(m) - d) <= 1e-13 * np.linalg.norm(d)
            assert np.linalg.norm(B.adjoint(rv) - gt) <= 1e-13 * np.linalg.norm(gt)
        with pytest.raises(ValueError):
            op.BCCB(K, g, Nmin_y - 1, Nmin_x)
