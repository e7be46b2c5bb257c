"""Local physics of the DDA: polarizability and the dyadic Green function.

Oracle (test infrastructure only).  Units follow the paper: Gaussian units,
time dependence exp(-i w t), polarizabilities without the voxel-volume factor
(Section 2.1, the remark after the LDR definition).
"""
from __future__ import annotations

import numpy as np

# Lattice-dispersion-relation constants exactly as printed in Section 2.1.
LDR_B1 = -1.891531
LDR_B2 = 0.1648469
LDR_B3 = -1.7700004


def alpha_cm(eps):
    """Clausius-Mossotti polarizability (3/4pi)(eps-1)/(eps+2) (Section 2.1)."""
    eps = np.asarray(eps, dtype=np.complex128)
    return 3.0 / (4.0 * np.pi) * (eps - 1.0) / (eps + 2.0)


def ldr_S(d, e):
    """S = sum_j (d_j e_j)^2 for unit direction d and polarisation e (Section 2.1)."""
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    return float(np.sum((d * e) ** 2))


def alpha_ldr(eps, k, dx, S):
    """LDR-corrected polarizability of Section 2.1.

    alpha = a_CM / (1 + a_CM [ (b1 + m^2 b2 + m^2 b3 S)(k dx)^2 - (2i/3)(k dx)^3 ])
    with m^2 = eps.
    """
    eps = np.asarray(eps, dtype=np.complex128)
    a = alpha_cm(eps)
    kd = k * dx
    corr = (LDR_B1 + eps * LDR_B2 + eps * LDR_B3 * S) * kd ** 2 - (2j / 3.0) * kd ** 3
    return a / (1.0 + a * corr)


def green_tensor(R, k):
    """Dyadic Green function g(R) of Section 2 (the definition after eq. 3).

    g = e^{ikr}/r [ k^2 (I - rr^T) + (ikr - 1)/r^2 (I - 3 rr^T) ],  r = |R|,
    rr^T the outer product of the unit vector (Algorithm 1 prints r^T r; the
    outer product is meant, as in the continuous definition).
    R has shape (..., 3) with no zero vector; returns (..., 3, 3) complex.
    """
    R = np.asarray(R, dtype=np.float64)
    r = np.sqrt(np.sum(R * R, axis=-1))
    rh = R / r[..., None]
    outer = rh[..., :, None] * rh[..., None, :]
    eye = np.eye(3)
    r_ = r[..., None, None]
    pref = np.exp(1j * k * r_) / r_
    return pref * (k * k * (eye - outer) + (1j * k * r_ - 1.0) / r_ ** 2 * (eye - 3.0 * outer))


def green_scalar(r, k):
    """Scalar outgoing Green function e^{ikr}/r whose (k^2 I + grad grad) is g."""
    return np.exp(1j * k * r) / r
