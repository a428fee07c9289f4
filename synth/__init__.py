"""Seeded synthetic inputs for the joint gravity-magnetic inversion workloads.

This module is shared by the tests, ``bench.py`` and the oracle checks.  It holds
*no arithmetic of the inversion method*: only geometry descriptions, seeded model
generators (blocky and smooth density / susceptibility distributions on a zero
background, the kind of bodies used in the paper's synthetic examples, Sec. 3) and
raw standard-normal draws.  Anything the method computes from these (kernels,
noise standard deviations of Eq. (noise), weights, the solve) is done separately by
the oracle and by the CUDA path.

Conventions (shared by both sides because they describe the input, not the math):
x = East, y = North, z = Down (metres).  Prism (r, iy, ix) spans
x in [x0 + ix*dx, x0 + (ix+1)*dx], y likewise, z in [z_edges[r], z_edges[r+1]].
Station (jy, jx) sits at the horizontal centre of prism column
(jy + off_y, jx + off_x) at height z = station_z (0 = the top of the first layer).
Model vectors are layer-major ``m[r][iy][ix]`` (ix fastest); data vectors are
``d[jy][jx]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np


@dataclass
class Grid:
    """Station grid and prism mesh of one geometry (Sec. 2.7.1)."""

    sx: int
    sy: int
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    z_edges: np.ndarray  # nz + 1 depths, metres, increasing (z positive down)
    station_z: float = 0.0
    off_x: int = 0
    off_y: int = 0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def s(self) -> int:
        return self.sx * self.sy


@dataclass
class Mag:
    """Inducing field: intensity (nT), inclination and declination (degrees)."""

    F: float = 50000.0
    incl: float = 60.0
    decl: float = 10.0


def uniform_grid(sx, sy, nx, ny, nz, cell, *, dz=None, off_x=0, off_y=0, station_z=0.0) -> Grid:
    dz = cell if dz is None else dz
    z = np.arange(nz + 1, dtype=np.float64) * dz
    return Grid(sx, sy, nx, ny, nz, float(cell), float(cell), z, station_z, off_x, off_y)


# ---------------------------------------------------------------------------
# model generators
# ---------------------------------------------------------------------------

def box_model(grid: Grid, boxes: List[Tuple[int, int, int, int, int, int]], value: float) -> np.ndarray:
    """Constant ``value`` inside inclusive index boxes (ix0, ix1, iy0, iy1, iz0, iz1)."""
    m = np.zeros((grid.nz, grid.ny, grid.nx))
    for ix0, ix1, iy0, iy1, iz0, iz1 in boxes:
        m[iz0:iz1 + 1, iy0:iy1 + 1, ix0:ix1 + 1] = value
    return m.reshape(-1)


def two_blocks(grid: Grid, value: float) -> np.ndarray:
    """Two blocks of constant contrast (the 16x16x8 small joint-inversion case)."""
    return box_model(grid, [(3, 6, 4, 9, 1, 3), (9, 12, 7, 12, 2, 5)], value)


def dipping_blocks(grid: Grid, value: float, seed: int, count: int = 3) -> np.ndarray:
    """``count`` parallelepipeds sheared one cell per layer, seeded extents."""
    rng = np.random.default_rng(seed)
    m = np.zeros((grid.nz, grid.ny, grid.nx))
    lo = max(2, min(grid.nx, grid.ny) // 12)
    hi = max(lo + 1, min(grid.nx, grid.ny) // 4)
    for _ in range(count):
        wx, wy = rng.integers(lo, hi + 1, size=2)
        top = int(rng.integers(1, max(2, grid.nz // 4)))
        thick = int(rng.integers(max(2, grid.nz // 8), max(3, grid.nz // 2)))
        x0 = int(rng.integers(0, max(1, grid.nx - wx - thick)))
        y0 = int(rng.integers(0, max(1, grid.ny - wy)))
        for r in range(top, min(grid.nz, top + thick)):
            sh = r - top
            m[r, y0:y0 + wy, min(grid.nx - 1, x0 + sh):min(grid.nx, x0 + sh + wx)] = value
    return m.reshape(-1)


def smooth_blocky(grid: Grid, vmax: float, seed: int, n_boxes: int = 6, sigma: float = 6.0) -> np.ndarray:
    """0.6 * smooth Gaussian-filtered field (rescaled to [0, 1]) + 0.4 * random boxes,
    clipped to [0, 1] and scaled by ``vmax``."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    g = rng.standard_normal((grid.nz, grid.ny, grid.nx))
    sm = gaussian_filter(g, sigma=(max(1.0, sigma * grid.nz / max(grid.nx, 1)), sigma, sigma), mode="wrap")
    sm = (sm - sm.min()) / max(sm.max() - sm.min(), 1e-30)
    bx = np.zeros_like(sm)
    for _ in range(n_boxes):
        wx, wy = rng.integers(max(2, grid.nx // 16), max(3, grid.nx // 4) + 1, size=2)
        wz = int(rng.integers(1, max(2, grid.nz // 3) + 1))
        x0 = int(rng.integers(0, grid.nx - wx + 1))
        y0 = int(rng.integers(0, grid.ny - wy + 1))
        z0 = int(rng.integers(0, grid.nz - wz + 1))
        bx[z0:z0 + wz, y0:y0 + wy, x0:x0 + wx] = 1.0
    return (np.clip(0.6 * sm + 0.4 * bx, 0.0, 1.0) * vmax).reshape(-1)


def uniform_model(grid: Grid, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=grid.n)


def standard_normal(shape, seed: int) -> np.ndarray:
    """Raw N(0, 1) draws, e.g. the unit noise that Eq. (noise) scales."""
    return np.random.default_rng(seed).standard_normal(shape)


# ---------------------------------------------------------------------------
# named workloads (shapes of the paper's synthetic examples, Sec. 3)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    grid: Grid
    mag: Mag
    m_true: Tuple[np.ndarray, np.ndarray]
    noise: Tuple[np.ndarray, np.ndarray]  # unit normal draws, one per field
    tau: Tuple[Tuple[float, float], Tuple[float, float]] = ((0.01, 0.01), (0.01, 0.01))
    extra: dict = field(default_factory=dict)


def small_joint(seed: int = 1) -> Workload:
    """16x16 stations, 16x16x8 cubes of 50 m; two correlated blocks."""
    g = uniform_grid(16, 16, 16, 16, 8, 50.0)
    m1 = two_blocks(g, 0.5)
    m2 = two_blocks(g, 0.05)
    e = standard_normal((2, g.s), seed)
    return Workload("joint-16x16x8", g, Mag(50000.0, 60.0, 10.0), (m1, m2), (e[0], e[1]))


def ragged_joint(seed: int = 6) -> Workload:
    """15x13 stations, 15x13x6 cubes of 50 m (13 rows per layer, not a multiple of
    four); smooth plus blocky models."""
    g = uniform_grid(15, 13, 15, 13, 6, 50.0)
    m1 = smooth_blocky(g, 0.5, seed, n_boxes=3, sigma=2.0)
    m2 = smooth_blocky(g, 0.05, seed + 1000, n_boxes=3, sigma=2.0)
    e = standard_normal((2, g.s), seed)
    return Workload("joint-15x13x6", g, Mag(50000.0, 60.0, 10.0), (m1, m2), (e[0], e[1]))


def odd_joint(seed: int = 7) -> Workload:
    """20x11 stations, 20x11x7 cubes of 50 m (an odd number of layers and of rows);
    smooth plus blocky models."""
    g = uniform_grid(20, 11, 20, 11, 7, 50.0)
    m1 = smooth_blocky(g, 0.5, seed, n_boxes=3, sigma=2.0)
    m2 = smooth_blocky(g, 0.05, seed + 1000, n_boxes=3, sigma=2.0)
    e = standard_normal((2, g.s), seed)
    return Workload("joint-20x11x7", g, Mag(50000.0, 60.0, 10.0), (m1, m2), (e[0], e[1]))


def operator_128(seed: int = 2) -> Workload:
    """128x128 stations, 128x128x32 cells of 50 m; smooth plus blocky models."""
    g = uniform_grid(128, 128, 128, 128, 32, 50.0)
    m1 = smooth_blocky(g, 1.0, seed)
    m2 = smooth_blocky(g, 0.1, seed + 1000)
    e = standard_normal((2, g.s), seed)
    return Workload("operator-128x128x32", g, Mag(50000.0, 60.0, 10.0), (m1, m2), (e[0], e[1]))


def joint_256(seed: int = 3, nz: int = 40, n: int = 256) -> Workload:
    """256x256 stations, 256x256x40 cells of 100 m; three dipping blocks."""
    g = uniform_grid(n, n, n, n, nz, 100.0)
    m1 = dipping_blocks(g, 1.0, seed)
    m2 = dipping_blocks(g, 0.1, seed)
    e = standard_normal((2, g.s), seed)
    return Workload(f"joint-{n}x{n}x{nz}", g, Mag(50000.0, 60.0, 10.0), (m1, m2), (e[0], e[1]))


def batched_sizes(seed: int = 4, count: int = 16):
    """Uneven (n, nz) pairs for the batched-inversion workload."""
    rng = np.random.default_rng(seed)
    sizes = []
    for _ in range(count):
        nx = int(rng.choice(np.arange(64, 257, 16)))
        ny = int(rng.choice(np.arange(64, 257, 16)))
        nz = int(rng.integers(16, 41))
        sizes.append((nx, ny, nz))
    return sizes
