"""Diagonal weights and the synthetic noise model (oracle; FP64).

Eq. (W): W = W_depth W_hard W_L1.  Eq. (WL): W_L1 = diag(((m - m_apr)^2 + eps^2)^(-1/4)),
the IRLS weight of the L1 stabiliser; the minimum-length variant (Sec. 3.1.5)
replaces it by the identity.  Both are the p = 1 and p = 2 cases of the exponent
(p - 2) / 4.  The depth weight of Sec. 2.1 is the standard Li & Oldenburg form,
whose exponent the paper does not print; here w_r = (z_r / z_1)^(-beta / 2) at the
layer centres z_r, so the top layer has weight 1.
Eq. (noise): sigma_j = tau1 |d_exact_j| + tau2 max |d_exact|, and W_d = diag(1 / sigma).
"""
from __future__ import annotations

import numpy as np


def depth_weights(z_edges, beta):
    zc = 0.5 * (np.asarray(z_edges[:-1]) + np.asarray(z_edges[1:]))
    return (zc / zc[0]) ** (-beta / 2.0)


def depth_weight_cells(z_edges, beta, nx, ny):
    """The depth weight broadcast to every cell of the layer-major model vector."""
    return np.repeat(depth_weights(z_edges, beta), nx * ny)


def lp_weight(m, m_apr, eps2, p):
    """Diagonal of W_L for the Lp stabiliser: ((m - m_apr)^2 + eps^2)^((p - 2) / 4)."""
    return ((np.asarray(m) - np.asarray(m_apr)) ** 2 + eps2) ** ((p - 2) / 4.0)


def noise_sigma(d_exact, tau1, tau2):
    d = np.abs(np.asarray(d_exact))
    return tau1 * d + tau2 * d.max()


def noisy_data(d_exact, tau1, tau2, unit_normal):
    """d_obs = d_exact + sigma * e for unit normal draws e."""
    sig = noise_sigma(d_exact, tau1, tau2)
    return np.asarray(d_exact) + sig * np.asarray(unit_normal), sig
