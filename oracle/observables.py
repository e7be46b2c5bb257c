"""Incident field and cross sections.

Oracle (test infrastructure only).  The paper's unknowns c are the
polarization per voxel (eqs. 7-10); the dipole moments are p = dx^3 c and the
Draine-Flatau polarizability is alpha_DF = dx^3 alpha (Section 2.1 notes the
paper drops the volume factor).  The paper prints no cross-section formula;
these are the standard DDA expressions of Draine & Flatau (the paper's DDA
reference) for a unit-amplitude incident wave (|e| = 1), Gaussian units:

    C_ext = 4 pi k sum_j Im(conj(E_inc,j) . p_j)
    C_abs = 4 pi k sum_j [ -Im(1/alpha_DF,j) - (2/3) k^3 ] |p_j|^2
    C_sca = 4 pi k sum_ij conj(p_i) . Im g(r_i - r_j) p_j,   Im g(0) = (2/3) k^3 I
          = k^4 * integral over the sphere of |n x (n x F(n))|^2,
            F(n) = sum_j p_j exp(-i k n . r_j).
For an exact solution C_ext = C_abs + C_sca (optical theorem).
"""
from __future__ import annotations

import numpy as np

from dda_inputs import voxel_centres
from .operator import comp_index, ice_positions
from .physics import green_tensor


def incident_field(mat: np.ndarray, dx: float, k: float, d, e) -> np.ndarray:
    """E_inc = e exp(i k d . r) on scatterer voxels, 0 on air; shape (3, n, m, l).

    Phase origin at the box centre (the paper does not state one).
    """
    n, m, l = mat.shape
    r = voxel_centres(l, m, n, dx)
    phase = np.exp(1j * k * (r @ np.asarray(d, dtype=np.float64)))
    ice = mat > 0
    out = np.asarray(e, dtype=np.float64)[:, None, None, None] * phase[None]
    return np.where(ice[None], out, 0.0).astype(np.complex128)


def c_ext(c_box, b_box, dx, k) -> float:
    p = dx ** 3 * c_box
    return float(4.0 * np.pi * k * np.sum(np.imag(np.conj(b_box) * p)))


def c_abs(c_box, mat, alpha_inv_vox, dx, k) -> float:
    p = dx ** 3 * c_box
    ice = mat > 0
    inv_df = alpha_inv_vox / dx ** 3
    p2 = np.sum(np.abs(p) ** 2, axis=0)
    val = (-np.imag(inv_df) - (2.0 / 3.0) * k ** 3) * p2
    return float(4.0 * np.pi * k * np.sum(val[ice]))


def c_sca_pairs(c_box, mat, dx, k) -> float:
    """C_sca by the double sum over voxel pairs (small problems)."""
    idx, r = ice_positions(mat, dx)
    p = dx ** 3 * c_box.reshape(3, -1)[:, idx].T          # (ni, 3)
    R = r[:, None, :] - r[None, :, :]
    diag = np.eye(len(r), dtype=bool)
    R[diag] = 1.0
    img = np.imag(green_tensor(R, k))
    img[diag] = (2.0 / 3.0) * k ** 3 * np.eye(3)
    val = np.einsum("ia,ijab,jb->", np.conj(p), img, p)
    return float(4.0 * np.pi * k * np.real(val))


def c_sca_fft(c_box, mat, dx, k) -> float:
    """Same quadratic form with Im g applied by a circulant-embedded FFT."""
    _, n, m, l = c_box.shape
    ice = mat > 0
    p = dx ** 3 * c_box * ice[None]
    zz, yy, xx = np.meshgrid(np.arange(2 * n), np.arange(2 * m), np.arange(2 * l), indexing="ij")
    off = lambda q, L: np.where(q < L, q, q - 2 * L)
    R = dx * np.stack([off(xx, l), off(yy, m), off(zz, n)], axis=-1).astype(np.float64)
    wrap = (xx == l) | (yy == m) | (zz == n)
    origin = (xx == 0) & (yy == 0) & (zz == 0)
    Rs = R.copy()
    Rs[origin] = 1.0
    img = np.imag(green_tensor(Rs, k))
    img[origin] = (2.0 / 3.0) * k ** 3 * np.eye(3)
    img[wrap] = 0.0
    pp = np.zeros((3, 2 * n, 2 * m, 2 * l), dtype=np.complex128)
    pp[:, :n, :m, :l] = p
    P = np.fft.fftn(pp, axes=(1, 2, 3))
    out = 0.0
    for a in range(3):
        Ya = np.zeros_like(P[0])
        for b in range(3):
            Ya += np.fft.fftn(img[..., a, b]) * P[b]
        ya = np.fft.ifftn(Ya)[:n, :m, :l]
        out += np.sum(np.conj(p[a]) * ya)
    return float(4.0 * np.pi * k * np.real(out))


def c_sca_farfield(c_box, mat, dx, k, n_theta: int = 48, n_phi: int = 96) -> float:
    """C_sca = k^4 integral |n x (n x F)|^2 dOmega (Gauss-Legendre in cos theta x uniform phi)."""
    idx, r = ice_positions(mat, dx)
    p = dx ** 3 * c_box.reshape(3, -1)[:, idx].T
    mu, w = np.polynomial.legendre.leggauss(n_theta)
    phi = 2 * np.pi * np.arange(n_phi) / n_phi
    total = 0.0
    for ct, wt in zip(mu, w):
        st = np.sqrt(max(0.0, 1.0 - ct * ct))
        nvec = np.stack([st * np.cos(phi), st * np.sin(phi), np.full_like(phi, ct)], axis=1)
        F = np.exp(-1j * k * nvec @ r.T) @ p                  # (n_phi, 3)
        Ft = F - nvec * np.sum(nvec * F, axis=1)[:, None]      # transverse part
        total += wt * (2 * np.pi / n_phi) * np.sum(np.abs(Ft) ** 2)
    return float(k ** 4 * total)
