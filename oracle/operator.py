"""Sensitivity operators of the gravity and magnetic problems (oracle; FP64).

Eq. (d=gm): d^(i) = A^(i) m^(i), A^(i) of size m x n, one column per prism and one
row per station, entries the closed-form prism fields of ``oracle.prism``.

Sec. 2.7.1 states that with stations on a uniform grid and a uniform mesh each
depth block A_(r) is BTTB, so an entry depends only on the layer r and on the
station-minus-prism index offsets (a, b).  That makes the dense product
computable exactly from a table of those unique entries; the FFT evaluation is
the same product, so the oracle of the operator is the product itself, written
as a plain sum.  ``BCCB`` states the paper's own evaluation of that product
(Sec. 2.7.1: per layer IFFT2(FFT2(T) . FFT2(X)), with numpy's FFT as the library
step), pinned against the plain sum; it lets the tests reach workloads whose
plain sums would take hours.

Index conventions: cell c = (r * ny + iy) * nx + ix, station j = jy * sx + jx,
a = (jy + off_y) - iy, b = (jx + off_x) - ix.
"""
from __future__ import annotations

import numpy as np

from .prism import FAR, cubature_order, prism_dT, prism_dT_cubature, prism_gz, prism_gz_cubature

GRAVITY = 1
MAGNETIC = 2


def _kernel(field, mag, x0, y0, z0, x1, x2, y1, y2, z1, z2):
    """The prism field for broadcast arrays of stations and prisms: the closed form
    (corner sums) near the station, cubature for prisms whose centre is at least FAR
    times their largest side away (where the corner sums cancel)."""
    if field not in (GRAVITY, MAGNETIC):
        raise ValueError(field)
    a = np.broadcast_arrays(*[np.asarray(v, dtype=np.float64) for v in (x0, y0, z0, x1, x2, y1, y2, z1, z2)])
    x0, y0, z0, x1, x2, y1, y2, z1, z2 = [v.reshape(-1) for v in a]
    size = np.maximum(np.maximum(x2 - x1, y2 - y1), z2 - z1)
    dist = np.sqrt((0.5 * (x1 + x2) - x0) ** 2 + (0.5 * (y1 + y2) - y0) ** 2 + (0.5 * (z1 + z2) - z0) ** 2)
    out = np.empty(x0.shape)
    near = dist < FAR * size
    args = lambda m: (x0[m], y0[m], z0[m], x1[m], x2[m], y1[m], y2[m], z1[m], z2[m])
    if field == GRAVITY:
        out[near] = prism_gz(*args(near))
    else:
        out[near] = prism_dT(*args(near), mag.F, mag.incl, mag.decl)
    order = np.where(near, 0, cubature_order(dist, size))
    for n in (5, 4, 3):
        m = order == n
        if not m.any():
            continue
        if field == GRAVITY:
            out[m] = prism_gz_cubature(*args(m), n=n)
        else:
            out[m] = prism_dT_cubature(*args(m), mag.F, mag.incl, mag.decl, n=n)
    return out.reshape(a[0].shape)


def station_xy(grid):
    """Horizontal station coordinates, shape (s,), (s,)."""
    jx = np.arange(grid.sx) + grid.off_x
    jy = np.arange(grid.sy) + grid.off_y
    X, Y = np.meshgrid((jx + 0.5) * grid.dx, (jy + 0.5) * grid.dy)
    return X.reshape(-1), Y.reshape(-1)


def dense_matrix(grid, field, mag=None) -> np.ndarray:
    """A (s x n): entry [j, c] = field at station j of prism c with unit property."""
    xs, ys = station_xy(grid)
    ix = np.arange(grid.nx)
    iy = np.arange(grid.ny)
    IX, IY = np.meshgrid(ix, iy)
    IX = IX.reshape(-1)
    IY = IY.reshape(-1)
    A = np.empty((grid.s, grid.n))
    layer = grid.nx * grid.ny
    for r in range(grid.nz):
        A[:, r * layer:(r + 1) * layer] = _kernel(
            field, mag,
            xs[:, None], ys[:, None], grid.station_z,
            (IX * grid.dx)[None, :], ((IX + 1) * grid.dx)[None, :],
            (IY * grid.dy)[None, :], ((IY + 1) * grid.dy)[None, :],
            grid.z_edges[r], grid.z_edges[r + 1])
    return A


def table_offsets(grid):
    """Ranges of the offsets a (rows) and b (columns) covered by the kernel table."""
    a = np.arange(grid.off_y - (grid.ny - 1), grid.off_y + grid.sy)
    b = np.arange(grid.off_x - (grid.nx - 1), grid.off_x + grid.sx)
    return a, b


def kernel_table(grid, field, mag=None) -> np.ndarray:
    """K[r, a - a_min, b - b_min] = field of prism (r, iy, ix) at station (jy, jx)
    for any pair with (jy + off_y - iy, jx + off_x - ix) = (a, b).

    The station sits at horizontal distance (b dx, a dy) from the prism centre,
    so the prism spans u in [-b dx - dx/2, -b dx + dx/2] and likewise in v.
    """
    a, b = table_offsets(grid)
    B, Aoff = np.meshgrid(b, a)
    K = np.empty((grid.nz, a.size, b.size))
    for r in range(grid.nz):
        K[r] = _kernel(field, mag, 0.0, 0.0, grid.station_z,
                       (-B - 0.5) * grid.dx, (-B + 0.5) * grid.dx,
                       (-Aoff - 0.5) * grid.dy, (-Aoff + 0.5) * grid.dy,
                       grid.z_edges[r], grid.z_edges[r + 1])
    return K


def forward_dense(A, m):
    return A @ m


def adjoint_dense(A, r):
    return A.T @ r


def _table_block(K, grid, jy, jx):
    """The (nz, ny, nx) block of table entries seen by station (jy, jx):
    entry [r, iy, ix] = K_r at offsets (jy + off_y - iy, jx + off_x - ix)."""
    a0 = grid.off_y - (grid.ny - 1)
    b0 = grid.off_x - (grid.nx - 1)
    ia = (jy + grid.off_y - np.arange(grid.ny)) - a0
    ib = (jx + grid.off_x - np.arange(grid.nx)) - b0
    return K[:, ia[:, None], ib[None, :]]


def forward_rows(K, grid, m, stations):
    """(A m)_j for the listed station indices j, as direct sums over all cells."""
    m3 = np.asarray(m, dtype=np.float64).reshape(grid.nz, grid.ny, grid.nx)
    out = np.empty(len(stations))
    for t, j in enumerate(stations):
        jy, jx = divmod(int(j), grid.sx)
        out[t] = np.sum(_table_block(K, grid, jy, jx) * m3)
    return out


def adjoint_cols(K, grid, rvec, cells):
    """(A^T r)_c for the listed cell indices c, as direct sums over all stations."""
    r2 = np.asarray(rvec, dtype=np.float64).reshape(grid.sy, grid.sx)
    a0 = grid.off_y - (grid.ny - 1)
    b0 = grid.off_x - (grid.nx - 1)
    out = np.empty(len(cells))
    layer = grid.nx * grid.ny
    for t, c in enumerate(cells):
        r, rem = divmod(int(c), layer)
        iy, ix = divmod(rem, grid.nx)
        ia = (np.arange(grid.sy) + grid.off_y - iy) - a0
        ib = (np.arange(grid.sx) + grid.off_x - ix) - b0
        out[t] = np.sum(K[r][ia[:, None], ib[None, :]] * r2)
    return out


def forward_direct(K, grid, m):
    """A m for every station (direct sums; O(s n))."""
    return forward_rows(K, grid, m, range(grid.s))


def adjoint_direct(K, grid, rvec):
    """A^T r for every cell (direct sums; O(s n))."""
    return adjoint_cols(K, grid, rvec, range(grid.n))


def dense_from_table(K, grid) -> np.ndarray:
    """The dense matrix assembled from the table (the BTTB structure of each depth
    block): A[j, c] = K[r, a - a_min, b - b_min] with (a, b) the index offsets of
    station j and cell c."""
    jy, jx = np.divmod(np.arange(grid.s), grid.sx)
    c = np.arange(grid.n)
    r, rem = np.divmod(c, grid.nx * grid.ny)
    iy, ix = np.divmod(rem, grid.nx)
    ia = (jy[:, None] + grid.off_y - iy[None, :]) - (grid.off_y - (grid.ny - 1))
    ib = (jx[:, None] + grid.off_x - ix[None, :]) - (grid.off_x - (grid.nx - 1))
    return K[r[None, :], ia, ib]


class BCCB:
    """The products of Sec. 2.7.1 through the circulant embedding: the table of layer r
    goes to T_r[c mod Ny, c' mod Nx] = K_r(c, c') for c in [-(ny-1), sy-1] (likewise in
    x), the model layer to the upper-left corner of an Ny x Nx zero array; the forward
    product is the upper-left sy x sx block of sum_r IFFT2(FFT2(T_r) FFT2(X_r)), the
    adjoint the upper-left ny x nx block of IFFT2(conj(FFT2(T_r)) FFT2(V)) per layer.
    Real transforms (numpy.fft.rfft2) since T, X and V are real.  FP64."""

    def __init__(self, K, grid, Ny, Nx):
        if Ny < grid.sy + grid.ny - 1 or Nx < grid.sx + grid.nx - 1:
            raise ValueError("padded size below s + n - 1")
        self.g, self.Ny, self.Nx = grid, Ny, Nx
        ia = np.arange(-(grid.ny - 1), grid.sy) % Ny
        ib = np.arange(-(grid.nx - 1), grid.sx) % Nx
        T = np.zeros((grid.nz, Ny, Nx))
        T[:, ia[:, None], ib[None, :]] = K
        self.Th = np.fft.rfft2(T)

    def forward(self, m):
        g = self.g
        X = np.zeros((g.nz, self.Ny, self.Nx))
        X[:, :g.ny, :g.nx] = np.asarray(m, dtype=np.float64).reshape(g.nz, g.ny, g.nx)
        Y = np.sum(self.Th * np.fft.rfft2(X), axis=0)
        return np.fft.irfft2(Y, s=(self.Ny, self.Nx))[:g.sy, :g.sx].reshape(-1)

    def adjoint(self, rvec):
        g = self.g
        V = np.zeros((self.Ny, self.Nx))
        V[:g.sy, :g.sx] = np.asarray(rvec, dtype=np.float64).reshape(g.sy, g.sx)
        Z = np.fft.irfft2(np.conj(self.Th) * np.fft.rfft2(V)[None], s=(self.Ny, self.Nx))
        return Z[:, :g.ny, :g.nx].reshape(-1)
