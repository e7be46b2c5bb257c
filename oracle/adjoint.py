"""Gradient of the extinction cross section with respect to each voxel's permittivity.

Oracle (test infrastructure only).  C_ext = 4 pi k dx^3 sum_j Im(conj(b_j) . c_j)
with A(eps) c = b.  Perturbing eps_j changes only the diagonal entry
alpha_j^{-1} (Section 2.1), so dc = -A^{-1} dA c and

    dC_ext = -4 pi k dx^3 Im( lambda^T dA c ),   A^T lambda = conj(b).

The DDA matrix is complex symmetric (A = A^T, Section 2.2), so lambda solves
A lambda = conj(b): the adjoint is a second solve with the same operator.
With g_j = (lambda_j . c_j) d(alpha_j^{-1})/d(eps_j) (unconjugated product over
the three components):

    dC_ext / d Re(eps_j) = -4 pi k dx^3 Im(g_j),
    dC_ext / d Im(eps_j) = -4 pi k dx^3 Re(g_j).

For the LDR polarizability 1/alpha = 1/alpha_CM + (b1 + eps b2 + eps b3 S)(k dx)^2
- (2i/3)(k dx)^3 and 1/alpha_CM = (4 pi/3)(eps + 2)/(eps - 1):

    d(1/alpha)/d eps = -4 pi/(eps - 1)^2 + (b2 + b3 S)(k dx)^2.
"""
from __future__ import annotations

import numpy as np

from . import observables, operator, physics


def dalpha_inv_deps(eps, k, dx, S):
    eps = np.asarray(eps, dtype=np.complex128)
    return -4.0 * np.pi / (eps - 1.0) ** 2 + (physics.LDR_B2 + physics.LDR_B3 * S) * (k * dx) ** 2


def ext_gradient(prob, c_box: np.ndarray, lam_box: np.ndarray) -> np.ndarray:
    """(2, n, m, l) real array: dC_ext/dRe(eps_j) and dC_ext/dIm(eps_j); zero on air."""
    mat = prob.mat
    eps_tab = np.zeros(len(prob.eps) + 1, dtype=np.complex128)
    eps_tab[1:] = prob.eps
    eps_vox = eps_tab[mat]
    d = np.where(mat > 0, dalpha_inv_deps(np.where(mat > 0, eps_vox, 2.0), prob.k, prob.dx, prob.S), 0.0)
    g = np.sum(lam_box * c_box, axis=0) * d
    pref = -4.0 * np.pi * prob.k * prob.dx ** 3
    return np.stack([pref * np.imag(g), pref * np.real(g)])


def adjoint_rhs(prob) -> np.ndarray:
    return np.conj(prob.rhs())


def c_ext_of(prob, c_box) -> float:
    return observables.c_ext(c_box, prob.rhs(), prob.dx, prob.k)
