"""Composite Gauss-Legendre cubature over a box (test helper, independent of the
closed forms it checks)."""
import numpy as np


def gl_box(fun, x1, x2, y1, y2, z1, z2, pts=16, sub=4):
    g, wg = np.polynomial.legendre.leggauss(pts)

    def nodes(a, b):
        edges = np.linspace(a, b, sub + 1)
        xs, ws = [], []
        for lo, hi in zip(edges[:-1], edges[1:]):
            xs.append(0.5 * (hi - lo) * g + 0.5 * (hi + lo))
            ws.append(0.5 * (hi - lo) * wg)
        return np.concatenate(xs), np.concatenate(ws)

    xs, wx = nodes(x1, x2)
    ys, wy = nodes(y1, y2)
    zs, wz = nodes(z1, z2)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
    return np.sum(fun(X, Y, Z) * W)
