"""Circulant approximations of the BTTB blocks and the circulant preconditioners.

Oracle (test infrastructure only).

* T. Chan's optimal circulant, eq. (13) (Section 3): for a Toeplitz matrix
  with T[i, j] = t_{i-j}, the Frobenius-nearest circulant has first column
      c_p = ((l - p) t_p + p t_{p-l}) / l,   0 <= p < l.
* Chan-Olkin (Section 3): applying eq. (13) level by level to a multilevel
  Toeplitz matrix gives the Frobenius-nearest multilevel circulant.  The
  paper applies it on x and y (the 2-level preconditioner of Section 3.1);
  applying it on all three levels gives the 3-level (block-circulant with
  3x3 blocks) preconditioner mentioned at the end of Section 3.2.
* Preconditioner (eq. 20, Section 3.1): P = alpha_tilde^{-1} I - dx^3 C, with
  alpha_tilde the polarizability of the scatterer's material ("ice").
* Strang's circulant, the alternative Section 3 names: keep the central
  diagonals of the Toeplitz matrix, c_p = t_p for p < l/2 and c_p = t_{p-l}
  for p > l/2; for even l the paper gives no rule at p = l/2, and the average
  (t_{l/2} + t_{-l/2}) / 2 is taken (it keeps each block's parity).

Each function here works from the Green function's values at signed offsets
(operator.signed_tensor), so no symmetry table is used; the brute-force
routine works from the dense matrix alone.
"""
from __future__ import annotations

import numpy as np

from dda_inputs import voxel_centres
from .operator import COMPONENTS, comp_index, signed_tensor
from .physics import green_tensor


def chan_1d(t_signed: np.ndarray) -> np.ndarray:
    """Eq. (13) for one Toeplitz matrix.

    t_signed has length 2l-1 with t_signed[o + l - 1] = t_o for offsets
    o = -(l-1) .. l-1.  Returns c_0 .. c_{l-1}.
    """
    L = (len(t_signed) + 1) // 2
    c = np.empty(L, dtype=np.complex128)
    for p in range(L):
        c[p] = (L - p) / L * t_signed[p + L - 1]
        if p > 0:
            c[p] += p / L * t_signed[p - L + L - 1]
    return c


def chan_axis(S: np.ndarray, axis: int) -> np.ndarray:
    """Apply eq. (13) along one axis of an array of signed offsets.

    The axis has length 2L-1 (offsets -(L-1)..L-1) on input and length L
    (circulant index 0..L-1) on output; other axes are left as they are.
    """
    S = np.moveaxis(S, axis, 0)
    L = (S.shape[0] + 1) // 2
    out = np.empty((L,) + S.shape[1:], dtype=np.complex128)
    for p in range(L):
        out[p] = (L - p) / L * S[p + L - 1]
        if p > 0:
            out[p] += p / L * S[p - L + L - 1]
    return np.moveaxis(out, 0, axis)


def strang_axis(S: np.ndarray, axis: int) -> np.ndarray:
    """Strang's circulant along one axis (same shapes as chan_axis)."""
    S = np.moveaxis(S, axis, 0)
    L = (S.shape[0] + 1) // 2
    out = np.empty((L,) + S.shape[1:], dtype=np.complex128)
    for p in range(L):
        if 2 * p < L:
            out[p] = S[p + L - 1]
        elif 2 * p > L:
            out[p] = S[p - L + L - 1]
        else:
            out[p] = 0.5 * (S[p + L - 1] + S[p - L + L - 1])
    return np.moveaxis(out, 0, axis)


def toeplitz_dense(t_signed: np.ndarray) -> np.ndarray:
    """Dense Toeplitz matrix T[i, j] = t_{i-j}."""
    L = (len(t_signed) + 1) // 2
    i, j = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    return t_signed[i - j + L - 1]


def circulant_dense(c: np.ndarray) -> np.ndarray:
    """Dense circulant matrix C[i, j] = c_{(i-j) mod l}."""
    L = len(c)
    i, j = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    return c[(i - j) % L]


def bttb_block_dense(l: int, m: int, n: int, dx: float, k: float, comp: int) -> np.ndarray:
    """Dense block G_comp over the whole box: T[i, j] = g_comp(r_i - r_j), zero diagonal.

    Voxels in flat (z, y, x) order.  Evaluated pair by pair from the Green
    function (no Toeplitz structure is assumed).
    """
    r = voxel_centres(l, m, n, dx).reshape(-1, 3)
    R = r[:, None, :] - r[None, :, :]
    diag = np.eye(len(r), dtype=bool)
    R[diag] = 1.0
    g = green_tensor(R, k)
    a, b = COMPONENTS[comp]
    T = g[:, :, a, b].copy()
    T[diag] = 0.0
    return T


def wrapped_average(T: np.ndarray, l: int, m: int, n: int,
                    wrap=(True, True, True)) -> np.ndarray:
    """Brute-force Frobenius-optimal multilevel circulant of a dense block.

    For every pair of voxels (i, j) form the offset d = r_i - r_j in voxel
    units; on a wrapped axis take d mod L, on an unwrapped axis keep d.
    The optimal coefficient for each (wrapped) offset is the mean of T over
    the pairs that share it.  Returns an array indexed
    [z-offset, y-offset, x-offset]; a wrapped axis has length L (0..L-1),
    an unwrapped one 2L-1 (offset + L - 1).
    """
    z, y, x = np.meshgrid(np.arange(n), np.arange(m), np.arange(l), indexing="ij")
    pos = np.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], axis=1)
    d = pos[:, None, :] - pos[None, :, :]
    dims = (l, m, n)
    keys = []
    shape = []
    for ax in range(3):
        L = dims[ax]
        if wrap[ax]:
            keys.append(d[..., ax] % L)
            shape.append(L)
        else:
            keys.append(d[..., ax] + L - 1)
            shape.append(2 * L - 1)
    flat = (keys[2] * shape[1] + keys[1]) * shape[0] + keys[0]
    size = shape[0] * shape[1] * shape[2]
    sums = np.bincount(flat.reshape(-1), weights=T.real.reshape(-1), minlength=size) \
        + 1j * np.bincount(flat.reshape(-1), weights=T.imag.reshape(-1), minlength=size)
    cnt = np.bincount(flat.reshape(-1), minlength=size)
    out = np.where(cnt > 0, sums / np.maximum(cnt, 1), 0.0)
    return out.reshape(shape[2], shape[1], shape[0])


def multilevel_circulant(l: int, m: int, n: int, dx: float, k: float,
                         levels=(True, True, True), kind: str = "chan") -> np.ndarray:
    """Closed-form multilevel circulant of all six blocks.

    Eq. (13) (kind "chan") or Strang's circulant (kind "strang") applied
    along each level marked True (x, y, z order).  Returns (6, nz, ny, nx)
    where a circulant level has length L and a Toeplitz one 2L-1 (signed
    offset + L - 1).
    """
    axis_op = {"chan": chan_axis, "strang": strang_axis}[kind]
    S = signed_tensor(l, m, n, dx, k)
    if levels[0]:
        S = axis_op(S, 3)
    if levels[1]:
        S = axis_op(S, 2)
    if levels[2]:
        S = axis_op(S, 1)
    return S


def assemble_3x3(six: np.ndarray) -> np.ndarray:
    """(6, ...) symmetric components -> (..., 3, 3)."""
    out = np.empty(six.shape[1:] + (3, 3), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            out[..., a, b] = six[comp_index(a, b)]
    return out


def precond3_lambda(l: int, m: int, n: int, dx: float, k: float,
                    alpha_tilde_inv: complex, kind: str = "chan") -> np.ndarray:
    """Per-frequency 3x3 symbol of the 3-level preconditioner, shape (n, m, l, 3, 3).

    Lambda(w) = alpha_tilde^{-1} I - dx^3 Chat(w), Chat = 3-D DFT of the
    3-level circulant's first column (a circulant is diagonalised by the DFT,
    Section 3).
    """
    C = multilevel_circulant(l, m, n, dx, k, (True, True, True), kind)
    Chat = np.fft.fftn(C, axes=(1, 2, 3))
    lam = -dx ** 3 * assemble_3x3(Chat)
    lam += alpha_tilde_inv * np.eye(3)
    return lam


def precond3_apply(v: np.ndarray, lam_inv: np.ndarray) -> np.ndarray:
    """z = P^{-1} v for the 3-level preconditioner; v is (3, n, m, l)."""
    V = np.fft.fftn(v, axes=(1, 2, 3))
    Z = np.einsum("zyxab,bzyx->azyx", lam_inv, V)
    return np.fft.ifftn(Z, axes=(1, 2, 3))


def precond3_dense(l: int, m: int, n: int, dx: float, k: float,
                   alpha_tilde_inv: complex) -> np.ndarray:
    """Dense P = alpha_tilde^{-1} I - dx^3 C over the box, unknowns (component, voxel).

    Assembled entry by entry from the 3-level circulant's first column with
    wrapped offsets: used to check the FFT form and the exactness of the
    preconditioner on a circulant system.
    """
    C = multilevel_circulant(l, m, n, dx, k, (True, True, True))
    z, y, x = np.meshgrid(np.arange(n), np.arange(m), np.arange(l), indexing="ij")
    x, y, z = x.reshape(-1), y.reshape(-1), z.reshape(-1)
    dxi = (x[:, None] - x[None, :]) % l
    dyi = (y[:, None] - y[None, :]) % m
    dzi = (z[:, None] - z[None, :]) % n
    nv = l * m * n
    P = np.zeros((3 * nv, 3 * nv), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            P[a * nv:(a + 1) * nv, b * nv:(b + 1) * nv] = -dx ** 3 * C[comp_index(a, b)][dzi, dyi, dxi]
    P += alpha_tilde_inv * np.eye(3 * nv)
    return P


def precond2_blocks(l: int, m: int, n: int, dx: float, k: float,
                    alpha_tilde_inv: complex, kind: str = "chan") -> np.ndarray:
    """Inverted dense blocks of the paper's 2-level preconditioner (Section 3.1).

    Circulant along x and y, Toeplitz along z.  After the 2-D DFT over
    (x, y) every frequency pair (wy, wx) carries a dense 3n x 3n block
    B[(a, z), (b, z')] = alpha_tilde^{-1} d_ab d_zz' - dx^3 Chat2_ab(z - z'; wy, wx)
    (eq. 19).  Returns the inverses, shape (m, l, 3n, 3n).
    """
    C2 = multilevel_circulant(l, m, n, dx, k, (True, True, False), kind)  # (6, 2n-1, m, l)
    Chat2 = np.fft.fftn(C2, axes=(2, 3))
    zi, zj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    off = zi - zj + n - 1
    blocks = np.zeros((m, l, 3 * n, 3 * n), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            c = comp_index(a, b)
            blk = Chat2[c][off]  # (n, n, m, l)
            blocks[:, :, a * n:(a + 1) * n, b * n:(b + 1) * n] = -dx ** 3 * np.moveaxis(blk, (0, 1), (2, 3))
    blocks += alpha_tilde_inv * np.eye(3 * n)
    return np.linalg.inv(blocks)


# The paper keeps z as the Toeplitz (dense) level of the 2-level preconditioner
# and notes that for long prisms making the long axis circulant may do better
# (Section 5).  Another Toeplitz level is reached by relabelling the axes
# cyclically so that it becomes z: a rotation of the frame, under which the
# Green tensor transforms as G(R r) = R G(r) R^T and the polarizability is
# unchanged, so the 2-level preconditioner of the relabelled box is the same
# operator.  Fields are (3, nz, ny, nx).
#   axis "x": (x', y', z') = (y, z, x), box (m, n, l)
#   axis "y": (x', y', z') = (z, x, y), box (n, l, m)
def toeplitz_frame_dims(l: int, m: int, n: int, axis: str):
    return {"z": (l, m, n), "x": (m, n, l), "y": (n, l, m)}[axis]


def to_toeplitz_frame(v: np.ndarray, axis: str) -> np.ndarray:
    if axis == "z":
        return v
    if axis == "x":
        return v[[1, 2, 0]].transpose(0, 3, 1, 2)
    return v[[2, 0, 1]].transpose(0, 2, 3, 1)


def from_toeplitz_frame(w: np.ndarray, axis: str) -> np.ndarray:
    if axis == "z":
        return w
    if axis == "x":
        return w[[2, 0, 1]].transpose(0, 2, 3, 1)
    return w[[1, 2, 0]].transpose(0, 3, 1, 2)


def precond2_apply(v: np.ndarray, blocks_inv: np.ndarray) -> np.ndarray:
    """z = P2^{-1} v: DFT over x and y, dense 3n block solve per (wy, wx), inverse DFT."""
    _, n, m, l = v.shape
    V = np.fft.fftn(v, axes=(2, 3))                     # (3, n, m, l)
    Vb = np.moveaxis(V, (2, 3), (0, 1)).reshape(m, l, 3 * n)
    Zb = np.einsum("yxij,yxj->yxi", blocks_inv, Vb)
    Z = np.moveaxis(Zb.reshape(m, l, 3, n), (0, 1), (2, 3))
    return np.fft.ifftn(Z, axes=(2, 3))
