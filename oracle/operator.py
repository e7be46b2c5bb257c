"""The DDA system matrix: Algorithm 1 tensor, dense assembly, FFT matvec.

Oracle (test infrastructure only).

System (Section 2.2, the block system after Algorithm 1):
    (alpha^{-1} - dx^3 G) c = E_inc
restricted to the scatterer's voxels (eq. 8: air voxels carry no
polarization).  G_ab(i, j) = g_ab(r_i - r_j) for i != j (midpoint rule,
eq. 12) and the self term is alpha_i^{-1} (eq. 11).

Box form.  The GPU works on the whole l x m x n box.  Reading of eq. 8: the
unknowns of air voxels are decoupled and their rows are alpha_tilde^{-1} c_a,
so the box matrix is block diagonal {scatterer block, alpha_tilde^{-1} I};
with a zero right-hand side on air the air unknowns solve to zero and the
scatterer block is exactly the matrix above.

Array layout: a field on the box is (3, n, m, l) complex (component, z, y,
x), x fastest, which is the voxel order of Algorithm 1.
"""
from __future__ import annotations

import numpy as np

from dda_inputs import voxel_centres
from .physics import green_tensor

# The six unique blocks in the order of Algorithm 1: xx, xy, xz, yy, yz, zz.
COMPONENTS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))


def comp_index(a: int, b: int) -> int:
    """Position of block (a, b) (or (b, a)) in COMPONENTS."""
    if a > b:
        a, b = b, a
    return COMPONENTS.index((a, b))


def alg1_tensor(l: int, m: int, n: int, dx: float, k: float) -> np.ndarray:
    """Defining tensor of Algorithm 1, shape (6, n, m, l).

    Entry [c, kz, jy, ix] = g_c(dx * (ix, jy, kz)), the interaction between
    the first voxel and voxel (ix, jy, kz); zero at the origin.
    """
    z, y, x = np.meshgrid(np.arange(n), np.arange(m), np.arange(l), indexing="ij")
    R = dx * np.stack([x, y, z], axis=-1).astype(np.float64)
    out = np.zeros((6, n, m, l), dtype=np.complex128)
    nz = (x + y + z) > 0
    g = green_tensor(R[nz], k)
    for c, (a, b) in enumerate(COMPONENTS):
        out[c][nz] = g[:, a, b]
    return out


def signed_tensor(l: int, m: int, n: int, dx: float, k: float) -> np.ndarray:
    """g at every signed offset, shape (6, 2n-1, 2m-1, 2l-1), zero at the origin.

    Entry [c, r + n-1, q + m-1, p + l-1] = g_c(dx * (p, q, r)).  Evaluated
    directly from the Green function at each signed offset, so no parity
    argument is involved.
    """
    z, y, x = np.meshgrid(np.arange(-(n - 1), n), np.arange(-(m - 1), m),
                          np.arange(-(l - 1), l), indexing="ij")
    R = dx * np.stack([x, y, z], axis=-1).astype(np.float64)
    out = np.zeros((6, 2 * n - 1, 2 * m - 1, 2 * l - 1), dtype=np.complex128)
    nz = (x != 0) | (y != 0) | (z != 0)
    g = green_tensor(R[nz], k)
    for c, (a, b) in enumerate(COMPONENTS):
        out[c][nz] = g[:, a, b]
    return out


def ice_positions(mat: np.ndarray, dx: float) -> tuple[np.ndarray, np.ndarray]:
    """Flat indices (into the (n, m, l) box) and centres of non-air voxels."""
    n, m, l = mat.shape
    idx = np.flatnonzero(mat.reshape(-1) > 0)
    r = voxel_centres(l, m, n, dx).reshape(-1, 3)[idx]
    return idx, r


def dense_matrix(mat: np.ndarray, alpha_inv_vox: np.ndarray, k: float, dx: float,
                 rows_per_chunk: int = 512) -> np.ndarray:
    """Dense scatterer-only matrix, unknown order (component, voxel).

    A[(a, i), (b, j)] = alpha_i^{-1} delta_ab delta_ij - dx^3 g_ab(r_i - r_j) (i != j).
    alpha_inv_vox is the per-voxel inverse polarizability on the (n, m, l) box.
    """
    idx, r = ice_positions(mat, dx)
    ni = len(idx)
    A = np.zeros((3 * ni, 3 * ni), dtype=np.complex128)
    ainv = alpha_inv_vox.reshape(-1)[idx]
    for i0 in range(0, ni, rows_per_chunk):
        i1 = min(ni, i0 + rows_per_chunk)
        R = r[i0:i1, None, :] - r[None, :, :]
        same = np.zeros((i1 - i0, ni), dtype=bool)
        same[np.arange(i1 - i0), np.arange(i0, i1)] = True
        R[same] = 1.0  # placeholder, overwritten below
        g = green_tensor(R, k)
        g[same] = 0.0
        for a in range(3):
            for b in range(3):
                A[a * ni + i0:a * ni + i1, b * ni:(b + 1) * ni] = -dx ** 3 * g[:, :, a, b]
    for a in range(3):
        A[a * ni + np.arange(ni), a * ni + np.arange(ni)] += ainv
    return A


def box_to_ice(c_box: np.ndarray, mat: np.ndarray) -> np.ndarray:
    """(3, n, m, l) box field -> (3*n_ice,) vector in (component, voxel) order."""
    idx = np.flatnonzero(mat.reshape(-1) > 0)
    return c_box.reshape(3, -1)[:, idx].reshape(-1)


def ice_to_box(v: np.ndarray, mat: np.ndarray) -> np.ndarray:
    """Inverse of box_to_ice, zero on air."""
    n, m, l = mat.shape
    idx = np.flatnonzero(mat.reshape(-1) > 0)
    out = np.zeros((3, n * m * l), dtype=np.complex128)
    out[:, idx] = v.reshape(3, -1)
    return out.reshape(3, n, m, l)


def circulant_generator(l: int, m: int, n: int, dx: float, k: float) -> np.ndarray:
    """Generator of the (2n, 2m, 2l) circulant embedding of the BTTB blocks.

    Index p in [0, 2l) stands for offset p when p < l, offset p - 2l when
    p > l; the wrap index p = l is zero (it couples no pair of box voxels).
    Same on every axis.  Shape (6, 2n, 2m, 2l).
    """
    S = signed_tensor(l, m, n, dx, k)

    def axis_map(L):
        src = np.zeros(2 * L, dtype=np.int64)
        valid = np.ones(2 * L, dtype=bool)
        for p in range(2 * L):
            if p < L:
                src[p] = p + (L - 1)
            elif p == L:
                valid[p] = False
            else:
                src[p] = p - 2 * L + (L - 1)
        return src, valid

    sx, vx = axis_map(l)
    sy, vy = axis_map(m)
    sz, vz = axis_map(n)
    out = S[:, sz][:, :, sy][:, :, :, sx]
    keep = vz[:, None, None] & vy[None, :, None] & vx[None, None, :]
    return out * keep[None]


def kernel_spectrum(l: int, m: int, n: int, dx: float, k: float) -> np.ndarray:
    """3-D DFT of the embedded generator, shape (6, 2n, 2m, 2l)."""
    return np.fft.fftn(circulant_generator(l, m, n, dx, k), axes=(1, 2, 3))


def convolve_G(x_box: np.ndarray, Ghat: np.ndarray) -> np.ndarray:
    """(G x)_i = sum_j g(r_i - r_j) x_j over the box (no diagonal), via the FFT.

    x_box (3, n, m, l); returns (3, n, m, l).
    """
    _, n, m, l = x_box.shape
    xp = np.zeros((3, 2 * n, 2 * m, 2 * l), dtype=np.complex128)
    xp[:, :n, :m, :l] = x_box
    X = np.fft.fftn(xp, axes=(1, 2, 3))
    Y = np.zeros_like(X)
    for a in range(3):
        for b in range(3):
            Y[a] += Ghat[comp_index(a, b)] * X[b]
    y = np.fft.ifftn(Y, axes=(1, 2, 3))
    return y[:, :n, :m, :l]


def fft_matvec(c_box: np.ndarray, mat: np.ndarray, alpha_inv_vox: np.ndarray,
               alpha_tilde_inv: complex, k: float, dx: float,
               Ghat: np.ndarray | None = None) -> np.ndarray:
    """Box-form matvec y = A c (scatterer rows by the FFT, air rows alpha_tilde^{-1} c)."""
    _, n, m, l = c_box.shape
    if Ghat is None:
        Ghat = kernel_spectrum(l, m, n, dx, k)
    ice = mat > 0
    conv = convolve_G(c_box * ice[None], Ghat)
    return np.where(ice[None], alpha_inv_vox[None] * c_box - dx ** 3 * conv,
                    alpha_tilde_inv * c_box)


def alpha_inv_box(mat: np.ndarray, alpha_per_material) -> np.ndarray:
    """Per-voxel alpha^{-1} on the box; air voxels get 0 (their rows use alpha_tilde)."""
    table = np.zeros(len(alpha_per_material) + 1, dtype=np.complex128)
    table[1:] = 1.0 / np.asarray(alpha_per_material, dtype=np.complex128)
    return table[mat]


def matvec_rows(c_box: np.ndarray, mat: np.ndarray, alpha_inv_vox: np.ndarray,
                alpha_tilde_inv: complex, k: float, dx: float, rows) -> np.ndarray:
    """Selected rows of the box-form matvec by direct summation (no FFT).

    rows: iterable of flat voxel indices into the (n, m, l) box.  Returns
    (len(rows), 3): (A c) at those voxels, summing g(r_i - r_j) c_j over every
    scatterer voxel j != i (eq. 12) and adding the diagonal (eq. 11); air rows
    are alpha_tilde^{-1} c.
    """
    idx, r = ice_positions(mat, dx)
    cj = c_box.reshape(3, -1)[:, idx].T                      # (n_ice, 3)
    n, m, l = mat.shape
    centres = voxel_centres(l, m, n, dx).reshape(-1, 3)
    out = np.zeros((len(rows), 3), dtype=np.complex128)
    flat_mat = mat.reshape(-1)
    ci = c_box.reshape(3, -1)
    for t, i in enumerate(rows):
        if flat_mat[i] == 0:
            out[t] = alpha_tilde_inv * ci[:, i]
            continue
        R = centres[i][None, :] - r
        self_ = np.all(R == 0.0, axis=1)
        R[self_] = 1.0
        g = green_tensor(R, k)
        g[self_] = 0.0
        out[t] = alpha_inv_vox.reshape(-1)[i] * ci[:, i] - dx ** 3 * np.einsum("jab,jb->a", g, cj)
    return out
