"""Parity of the CUDA BTTB/FFT products (gj_g_forward, gj_g_adjoint; Sec. 2.7.1)
with the FP64 dense oracle (Eq. d=gm), through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import operator as oop
from tests.gpu_common import TOL, lib, rel, to_dev

pytestmark = pytest.mark.gpu

MAG = synth.Mag(50000.0, 60.0, 10.0)


def _grid(sx, sy, nx, ny, nz, dx=50.0, dy=None, dz=None, off=(0, 0), station_z=0.0, zvar=False):
    g = synth.uniform_grid(sx, sy, nx, ny, nz, dx, dz=dz, off_x=off[0], off_y=off[1], station_z=station_z)
    if dy is not None:
        g.dy = dy
    if zvar:
        g.z_edges = np.concatenate([[0.0], np.cumsum(np.linspace(20.0, 80.0, nz))])
    return g


CASES = {
    "joint16": (_grid(16, 16, 16, 16, 8), (0, 0)),
    "ragged": (_grid(13, 11, 13, 11, 5, dx=30.0), (0, 0)),
    "padding_prisms": (_grid(9, 7, 12, 10, 3, dx=40.0, dy=55.0, dz=30.0, off=(2, 1)), (0, 0)),
    "radix_3_5_17": (_grid(8, 8, 8, 8, 3), (15, 17)),
    "radix_11_13": (_grid(8, 8, 8, 8, 2), (22, 26)),
    "radix_7_odd": (_grid(10, 9, 10, 9, 2), (21, 49)),
    "lifted_varz": (_grid(12, 12, 12, 12, 6, station_z=-15.0, zvar=True), (0, 0)),
    "one_cell": (_grid(1, 1, 1, 1, 1), (0, 0)),
    "one_row": (_grid(7, 1, 7, 1, 4), (0, 0)),
    "column": (_grid(1, 6, 1, 6, 2), (0, 0)),
    # 512 x 512 embeddings: the specialised kernels serve the FP32 operators
    "fast512_small": (_grid(16, 16, 16, 16, 3), (512, 512)),
    "fast512_ragged": (_grid(13, 11, 20, 9, 2, dx=40.0, dy=55.0, off=(3, 0)), (512, 512)),
    "fast512_odd_lines": (_grid(7, 5, 7, 5, 5, station_z=-8.0, zvar=True), (512, 512)),
    # 256-row embeddings (N_y = 256, N_x = 512): the specialised kernels with
    # half-warp column transforms over layer pairs (odd layer counts leave one half idle)
    "fast256_small": (_grid(16, 16, 16, 16, 3), (256, 512)),
    "fast256_ragged": (_grid(13, 11, 20, 9, 2, dx=40.0, dy=55.0, off=(3, 0)), (256, 512)),
    "fast256_odd_lines": (_grid(7, 5, 7, 5, 5, station_z=-8.0, zvar=True), (256, 512)),
    "fast256_offset_y": (_grid(9, 12, 9, 10, 4, dx=30.0, off=(0, 2)), (256, 512)),
    # N_y = 1024: the warp-FFT column kernels behind the general row kernels (any N_x)
    "cols1024_small": (_grid(16, 16, 16, 16, 3), (1024, 32)),
    "cols1024_ragged": (_grid(13, 11, 20, 9, 2, dx=40.0, dy=55.0, off=(3, 0)), (1024, 36)),
    "cols1024_odd_lines": (_grid(7, 5, 7, 5, 5, station_z=-8.0, zvar=True), (1024, 15)),
    "cols1024_wide": (_grid(30, 6, 24, 6, 2, dx=20.0), (1024, 1024)),
    # N_x = 1024 as well: the warp-FFT row kernels of the same file
    "rows1024_ragged": (_grid(13, 11, 20, 9, 3, dx=40.0, dy=55.0, off=(3, 0)), (1024, 1024)),
    "rows1024_odd": (_grid(7, 5, 7, 5, 5, station_z=-8.0, zvar=True), (1024, 1024)),
}

FAST = {(512, 512), (256, 512)}


def fast_kind(prec, npad):
    """gj_op_info_t.fast_path expected for a padded size."""
    if prec != "fp32":
        return 0
    return 1 if npad in FAST else (2 if npad[0] == 1024 else 0)


@pytest.fixture(scope="module")
def gj():
    return lib()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("field", ["gravity", "magnetic"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_products_match_dense_oracle(gj, case, field, prec):
    g, npad = CASES[case]
    f = oop.GRAVITY if field == "gravity" else oop.MAGNETIC
    A = oop.dense_matrix(g, f, MAG)
    op = gj.bttb_setup(g, field, MAG if field == "magnetic" else None, precision=prec, npad=npad)
    assert op.info.fast_path == fast_kind(prec, npad)
    rng = np.random.default_rng(11)
    for trial in range(2):
        m = rng.uniform(0.0, 1.0, g.n) if trial == 0 else rng.standard_normal(g.n)
        r = rng.standard_normal(g.s)
        d = op.forward(to_dev(m, prec)).cpu().numpy()
        a = op.adjoint(to_dev(r, prec)).cpu().numpy()
        assert rel(d, A @ m) <= TOL[prec], (case, field, prec, rel(d, A @ m))
        assert rel(a, A.T @ r) <= TOL[prec], (case, field, prec, rel(a, A.T @ r))
    op.close()


def test_padded_size_does_not_change_the_product(gj):
    g = _grid(8, 8, 8, 8, 3)
    A = oop.dense_matrix(g, oop.MAGNETIC, MAG)
    m = np.random.default_rng(2).standard_normal(g.n)
    for npad in [(15, 15), (16, 16), (18, 20), (24, 27), (30, 25), (32, 64)]:
        op = gj.bttb_setup(g, "magnetic", MAG, precision="fp64", npad=npad)
        assert op.info.Ny == npad[0] and op.info.Nx == npad[1]
        assert rel(op.forward(to_dev(m, "fp64")).cpu().numpy(), A @ m) <= 1e-10


def test_invalid_arguments_raise(gj):
    g = _grid(8, 8, 8, 8, 3)
    with pytest.raises(gj.GJError):
        gj.bttb_setup(g, "gravity", npad=(14, 15))  # below s + n - 1
    with pytest.raises(gj.GJError):
        gj.bttb_setup(g, "gravity", npad=(19 * 1, 19))  # prime factor 19
    with pytest.raises(gj.GJError):
        gj.bttb_setup(g, "magnetic", None)
    bad = _grid(8, 8, 8, 8, 3, station_z=10.0)
    with pytest.raises(gj.GJError):
        gj.bttb_setup(bad, "gravity")


@pytest.fixture(scope="module")
def c2_tables():
    w = synth.operator_128()
    return w, {oop.GRAVITY: oop.kernel_table(w.grid, oop.GRAVITY), oop.MAGNETIC: oop.kernel_table(w.grid, oop.MAGNETIC, w.mag)}


@pytest.mark.parametrize("npad", [(255, 255), (0, 0)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_operator_128_sampled_rows(gj, c2_tables, npad, prec):
    """128x128 stations, 128x128x32 cells; padded 255x255 (3*5*17) and the autotuned size."""
    w, K = c2_tables
    g = w.grid
    rng = np.random.default_rng(5)
    st = np.unique(np.concatenate([[0, g.s - 1, g.sx - 1, g.s - g.sx], rng.integers(0, g.s, 40)]))
    cells = np.unique(np.concatenate([[0, g.n - 1], rng.integers(0, g.n, 40)]))
    r = rng.standard_normal(g.s)
    for f, name in [(oop.GRAVITY, "gravity"), (oop.MAGNETIC, "magnetic")]:
        op = gj.bttb_setup(g, name, w.mag if name == "magnetic" else None, precision=prec, npad=npad)
        m = w.m_true[0] if f == oop.GRAVITY else w.m_true[1]
        d = op.forward(to_dev(m, prec)).cpu().numpy()
        a = op.adjoint(to_dev(r, prec)).cpu().numpy()
        d_ref = oop.forward_rows(K[f], g, m, st)
        a_ref = oop.adjoint_cols(K[f], g, r, cells)
        tol = TOL[prec]  # relative L2 over the sampled outputs
        assert rel(d[st], d_ref) <= tol, (name, rel(d[st], d_ref))
        assert rel(a[cells], a_ref) <= tol, (name, rel(a[cells], a_ref))
        op.close()


def test_operator_128_adjoint_identity_fp64(gj, c2_tables):
    w, _ = c2_tables
    g = w.grid
    rng = np.random.default_rng(8)
    for name in ("gravity", "magnetic"):
        op = gj.bttb_setup(g, name, w.mag if name == "magnetic" else None, precision="fp64")
        m = rng.standard_normal(g.n)
        r = rng.standard_normal(g.s)
        d = op.forward(to_dev(m, "fp64")).cpu().numpy()
        a = op.adjoint(to_dev(r, "fp64")).cpu().numpy()
        lhs, rhs = d @ r, m @ a
        assert abs(lhs - rhs) <= 1e-12 * np.sqrt((d @ d) * (r @ r)), (name, lhs, rhs)
        op.close()


@pytest.fixture(scope="module")
def c3_tables():
    w = synth.joint_256()
    return w, {oop.GRAVITY: oop.kernel_table(w.grid, oop.GRAVITY),
               oop.MAGNETIC: oop.kernel_table(w.grid, oop.MAGNETIC, w.mag)}


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_joint_256_sampled_rows(gj, c3_tables, prec):
    """256x256 stations, 256x256x40 cells of 100 m, padded 512x512 (the benchmark
    workload): sampled forward rows and adjoint cells against direct sums."""
    w, K = c3_tables
    g = w.grid
    rng = np.random.default_rng(6)
    st = np.unique(np.concatenate([[0, g.s - 1, g.sx - 1, g.s - g.sx, g.s // 2 + 77], rng.integers(0, g.s, 24)]))
    cells = np.unique(np.concatenate([[0, g.n - 1, g.nx * g.ny - 1], rng.integers(0, g.n, 40)]))
    r = rng.standard_normal(g.s)
    for f, name in [(oop.GRAVITY, "gravity"), (oop.MAGNETIC, "magnetic")]:
        op = gj.bttb_setup(g, name, w.mag if name == "magnetic" else None, precision=prec)
        assert op.info.Nx == 512 and op.info.Ny == 512
        assert op.info.fast_path == (1 if prec == "fp32" else 0)
        m = w.m_true[0] if f == oop.GRAVITY else w.m_true[1]
        d = op.forward(to_dev(m, prec)).cpu().numpy()
        a = op.adjoint(to_dev(r, prec)).cpu().numpy()
        d_ref = oop.forward_rows(K[f], g, m, st)
        a_ref = oop.adjoint_cols(K[f], g, r, cells)
        # relative L2 over the sampled outputs (both sides integrate far prisms by
        # cubature, where the corner sums would cancel)
        tol_d = TOL[prec]
        tol_a = TOL[prec]
        assert rel(d[st], d_ref) <= tol_d, (name, rel(d[st], d_ref))
        assert rel(a[cells], a_ref) <= tol_a, (name, rel(a[cells], a_ref))
        print(f"\n256x256x40 {prec} {name}: sampled forward rel {rel(d[st], d_ref):.2e}, "
              f"sampled adjoint rel {rel(a[cells], a_ref):.2e}")
        # repeated calls give the same result: the persistent column kernel's
        # layer-sum partials and counters start clean each time and its sums run in
        # a fixed order (the generic kernels sum layers with atomics: rounding only)
        d2 = op.forward(to_dev(m, prec)).cpu().numpy()
        if op.info.fast_path:
            assert np.array_equal(d, d2)
        else:
            assert rel(d2, d) <= 1e-14
        op.close()


@pytest.mark.parametrize("case", ["fast512_small", "fast512_ragged", "joint16", "fast256_ragged", "fast256_odd_lines",
                                  "cols1024_ragged", "cols1024_odd_lines", "cols1024_wide"])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pair_products_match_dense_oracle(gj, case, prec):
    """gj_g_forward_pair / gj_g_adjoint_pair: both fields in one call (one set of joint
    launches on the fast path, two single-field calls otherwise) against the dense
    oracle and against the single-field calls."""
    g, npad = CASES[case]
    A = [oop.dense_matrix(g, oop.GRAVITY, MAG), oop.dense_matrix(g, oop.MAGNETIC, MAG)]
    ops = [gj.bttb_setup(g, "gravity", None, precision=prec, npad=npad),
           gj.bttb_setup(g, "magnetic", MAG, precision=prec, npad=npad)]
    rng = np.random.default_rng(41)
    m = [rng.uniform(0.0, 1.0, g.n), rng.standard_normal(g.n)]
    r = [rng.standard_normal(g.s), rng.standard_normal(g.s)]
    d = gj.g_forward_pair(ops, [to_dev(x, prec) for x in m])
    a = gj.g_adjoint_pair(ops, [to_dev(x, prec) for x in r])
    for i in range(2):
        di, ai = d[i].cpu().numpy(), a[i].cpu().numpy()
        assert rel(di, A[i] @ m[i]) <= TOL[prec], (case, i, rel(di, A[i] @ m[i]))
        assert rel(ai, A[i].T @ r[i]) <= TOL[prec], (case, i, rel(ai, A[i].T @ r[i]))
        ds = ops[i].forward(to_dev(m[i], prec)).cpu().numpy()
        as_ = ops[i].adjoint(to_dev(r[i], prec)).cpu().numpy()
        tol = 1e-13 if prec == "fp64" else 1e-6
        assert rel(di, ds) <= tol and rel(ai, as_) <= tol
    with pytest.raises(ValueError):
        gj.g_forward_pair([ops[0], ops[0]], [to_dev(x, prec) for x in m])


@pytest.mark.parametrize("shape", [(96, 128, 7), (128, 128, 6), (200, 100, 9)])
def test_fast256_largest_columns_sampled_rows(gj, shape):
    """N_y = 256 at its limits (up to 128 stations and prisms per column, odd and even
    layer counts, 100 m cells): sampled forward rows and adjoint cells against direct
    sums, and the same products through the 512 x 512 kernels."""
    nx, ny, nz = shape
    g = synth.uniform_grid(nx, ny, nx, ny, nz, 100.0)
    rng = np.random.default_rng(12)
    st = np.unique(np.concatenate([[0, g.s - 1, g.sx - 1, g.s - g.sx], rng.integers(0, g.s, 24)]))
    cells = np.unique(np.concatenate([[0, g.n - 1, g.nx * g.ny - 1], rng.integers(0, g.n, 40)]))
    m = synth.smooth_blocky(g, 1.0, seed=3)
    r = rng.standard_normal(g.s)
    for f, name in [(oop.GRAVITY, "gravity"), (oop.MAGNETIC, "magnetic")]:
        K = oop.kernel_table(g, f, MAG) if f == oop.MAGNETIC else oop.kernel_table(g, f)
        op = gj.bttb_setup(g, name, MAG if name == "magnetic" else None, precision="fp32", npad=(256, 512))
        assert op.info.fast_path == 1 and op.info.Ny == 256
        d = op.forward(to_dev(m, "fp32")).cpu().numpy()
        a = op.adjoint(to_dev(r, "fp32")).cpu().numpy()
        assert rel(d[st], oop.forward_rows(K, g, m, st)) <= TOL["fp32"], name
        assert rel(a[cells], oop.adjoint_cols(K, g, r, cells)) <= TOL["fp32"], name
        op512 = gj.bttb_setup(g, name, MAG if name == "magnetic" else None, precision="fp32", npad=(512, 512))
        assert rel(d, op512.forward(to_dev(m, "fp32")).cpu().numpy()) <= 1e-6
        assert rel(a, op512.adjoint(to_dev(r, "fp32")).cpu().numpy()) <= 1e-6
        op.close()
        op512.close()


def test_fast256_needs_room_for_the_columns(gj):
    """More than 128 stations or prisms per column keep N_y = 256 on the general
    kernels, with the same products as the 512 x 512 kernels."""
    m_seed = 4
    for sy, ny in [(129, 120), (100, 129)]:
        g = synth.uniform_grid(16, sy, 16, ny, 2, 50.0)
        op = gj.bttb_setup(g, "gravity", precision="fp32", npad=(256, 512))
        assert op.info.fast_path == 0
        ref = gj.bttb_setup(g, "gravity", precision="fp32", npad=(512, 512))
        assert ref.info.fast_path == 1
        m = synth.smooth_blocky(g, 1.0, seed=m_seed)
        assert rel(op.forward(to_dev(m, "fp32")).cpu().numpy(), ref.forward(to_dev(m, "fp32")).cpu().numpy()) <= 1e-6
        op.close()
        ref.close()


@pytest.mark.parametrize("shape", [(96, 512, 5), (512, 64, 3), (300, 260, 4)])
def test_cols1024_largest_columns_sampled_rows(gj, shape):
    """N_y = 1024 at its limits (up to 512 stations and prisms per column, 100 m cells):
    sampled forward rows and adjoint cells against direct sums, FP32 against FP64."""
    nx, ny, nz = shape
    g = synth.uniform_grid(nx, ny, nx, ny, nz, 100.0)
    rng = np.random.default_rng(13)
    st = np.unique(np.concatenate([[0, g.s - 1, g.sx - 1, g.s - g.sx], rng.integers(0, g.s, 24)]))
    cells = np.unique(np.concatenate([[0, g.n - 1, g.nx * g.ny - 1], rng.integers(0, g.n, 40)]))
    m = synth.uniform_model(g, 0.0, 1.0, seed=3)
    r = rng.standard_normal(g.s)
    Nx = {96: 192, 512: 1024, 300: 600}[nx]
    for f, name in [(oop.GRAVITY, "gravity"), (oop.MAGNETIC, "magnetic")]:
        K = oop.kernel_table(g, f, MAG) if f == oop.MAGNETIC else oop.kernel_table(g, f)
        op = gj.bttb_setup(g, name, MAG if name == "magnetic" else None, precision="fp32", npad=(1024, Nx))
        assert op.info.fast_path == 2 and op.info.Ny == 1024
        d = op.forward(to_dev(m, "fp32")).cpu().numpy()
        a = op.adjoint(to_dev(r, "fp32")).cpu().numpy()
        assert rel(d[st], oop.forward_rows(K, g, m, st)) <= TOL["fp32"], name
        assert rel(a[cells], oop.adjoint_cols(K, g, r, cells)) <= TOL["fp32"], name
        op64 = gj.bttb_setup(g, name, MAG if name == "magnetic" else None, precision="fp64", npad=(1024, Nx))
        assert rel(d, op64.forward(to_dev(m, "fp64")).cpu().numpy()) <= 1e-6
        assert rel(a, op64.adjoint(to_dev(r, "fp64")).cpu().numpy()) <= 1e-6
        op.close()
        op64.close()
