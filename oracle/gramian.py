"""The Gramian coupling constraint (oracle; FP64).

Eq. (Gramian): S_G(m1, m2) is the determinant of the 2 x 2 Gram matrix of the two
model vectors under the L2 inner product.  RRCG:2-3 give the ascent directions in
the original (unweighted) space: l1 = ||m2||^2 m1 - (m1, m2) m2 and
l2 = ||m1||^2 m2 - (m1, m2) m1 (half the gradient of S_G).  Eq. (steepestascenta/b)
give the same expressions for the weighted vectors (the weighted-space variant,
Sec. 3.1.4, Appendix A).
"""
from __future__ import annotations

import numpy as np


def gram_matrix(m1, m2):
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    return np.array([[m1 @ m1, m1 @ m2], [m2 @ m1, m2 @ m2]])


def gramian(m1, m2):
    """S_G = det of the Gram matrix."""
    g = gram_matrix(m1, m2)
    return g[0, 0] * g[1, 1] - g[0, 1] * g[1, 0]


def ascent_directions(m1, m2):
    """(l_G^(1), l_G^(2)) of RRCG:2-3 (equivalently Eq. steepestascenta/b)."""
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    a11 = m1 @ m1
    a22 = m2 @ m2
    a12 = m1 @ m2
    return a22 * m1 - a12 * m2, a11 * m2 - a12 * m1
