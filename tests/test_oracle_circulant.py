"""Pins of the oracle's circulant approximations (eq. 13, Section 3) and preconditioners."""
import numpy as np
import pytest

from dda_inputs import random_field
from oracle import circulant, krylov, operator


def test_chan_1d_equals_wrapped_diagonal_mean():
    rng = np.random.default_rng(0)
    for L in (1, 2, 5, 8):
        t = random_field(2 * L - 1, rng)
        T = circulant.toeplitz_dense(t)
        brute = circulant.wrapped_average(T, L, 1, 1)[0, 0]
        assert np.allclose(circulant.chan_1d(t), brute, rtol=1e-14, atol=1e-15)


def test_chan_1d_fixed_point_on_circulant():
    rng = np.random.default_rng(1)
    L = 7
    c = random_field(L, rng)
    # the Toeplitz symbol of a circulant: t_o = c_{o mod L}
    t = np.array([c[o % L] for o in range(-(L - 1), L)])
    assert np.allclose(circulant.chan_1d(t), c, rtol=1e-14, atol=0)
    assert np.allclose(circulant.circulant_dense(c), circulant.toeplitz_dense(t))


def test_chan_1d_is_frobenius_optimal():
    rng = np.random.default_rng(2)
    L = 6
    t = random_field(2 * L - 1, rng)
    T = circulant.toeplitz_dense(t)
    C = circulant.circulant_dense(circulant.chan_1d(t))
    best = np.linalg.norm(T - C)
    for _ in range(20):
        E = circulant.circulant_dense(random_field(L, rng))
        assert np.linalg.norm(T - (C + 1e-3 * E)) > best


def test_chan_1d_closed_form_values():
    # eq. (13) written out for L = 3: c0 = t0, c1 = (2 t1 + t_{-2})/3, c2 = (t2 + 2 t_{-1})/3
    t = {-2: 1.0 + 2j, -1: -0.5j, 0: 3.0, 1: 0.25, 2: -1.0 + 1j}
    arr = np.array([t[o] for o in range(-2, 3)])
    c = circulant.chan_1d(arr)
    assert np.allclose(c, [t[0], (2 * t[1] + t[-2]) / 3, (t[2] + 2 * t[-1]) / 3], rtol=1e-15)


@pytest.mark.parametrize("comp", range(6))
def test_multilevel_closed_form_equals_bruteforce(comp):
    l, m, n, dx, k = 4, 5, 6, 0.3, 1.7
    T = circulant.bttb_block_dense(l, m, n, dx, k, comp)
    closed3 = circulant.multilevel_circulant(l, m, n, dx, k, (True, True, True))[comp]
    brute3 = circulant.wrapped_average(T, l, m, n, (True, True, True))
    assert np.allclose(closed3, brute3, rtol=1e-12, atol=1e-13 * np.abs(brute3).max())
    closed2 = circulant.multilevel_circulant(l, m, n, dx, k, (True, True, False))[comp]
    brute2 = circulant.wrapped_average(T, l, m, n, (True, True, False))
    assert np.allclose(closed2, brute2, rtol=1e-12, atol=1e-13 * np.abs(brute2).max())


def test_precond3_fft_form_matches_dense_and_inverts():
    l, m, n, dx, k = 4, 3, 5, 0.4, 1.5
    ati = 20.0 - 0.3j
    P = circulant.precond3_dense(l, m, n, dx, k, ati)
    lam = circulant.precond3_lambda(l, m, n, dx, k, ati)
    lam_inv = np.linalg.inv(lam)
    assert np.allclose(np.einsum("...ab,...bc->...ac", lam, lam_inv), np.eye(3), atol=1e-12)
    rng = np.random.default_rng(3)
    v = random_field((3, n, m, l), rng)
    Pv = (P @ v.reshape(-1)).reshape(v.shape)
    # BCCB: P v computed with the symbol equals the dense product
    Pv_fft = np.fft.ifftn(np.einsum("zyxab,bzyx->azyx", lam, np.fft.fftn(v, axes=(1, 2, 3))), axes=(1, 2, 3))
    assert np.allclose(Pv_fft, Pv, rtol=1e-12, atol=1e-12 * np.abs(Pv).max())
    z = circulant.precond3_apply(Pv, lam_inv)
    assert np.allclose(z, v, rtol=1e-11, atol=1e-11)


def test_precond3_exact_on_circulant_system():
    # When the system matrix is itself the 3-level circulant, P^{-1} A = I:
    # right-preconditioned GMRES converges in one iteration.
    l, m, n, dx, k = 4, 4, 3, 0.5, 1.2
    ati = 15.0 + 0.0j
    P = circulant.precond3_dense(l, m, n, dx, k, ati)
    lam_inv = np.linalg.inv(circulant.precond3_lambda(l, m, n, dx, k, ati))
    rng = np.random.default_rng(4)
    b = random_field((3, n, m, l), rng)
    x, info = krylov.gmres(lambda v: (P @ v.reshape(-1)).reshape(v.shape), b, tol=1e-10,
                           restart=20, precond=lambda v: circulant.precond3_apply(v, lam_inv))
    assert info["converged"] and info["iters"] == 1


def test_precond2_blocks_invert_dense_2level():
    l, m, n, dx, k = 3, 4, 3, 0.5, 1.4
    ati = 18.0 - 0.2j
    C2 = circulant.multilevel_circulant(l, m, n, dx, k, (True, True, False))
    z, y, x = np.meshgrid(np.arange(n), np.arange(m), np.arange(l), indexing="ij")
    x, y, z = x.reshape(-1), y.reshape(-1), z.reshape(-1)
    dxi = (x[:, None] - x[None, :]) % l
    dyi = (y[:, None] - y[None, :]) % m
    dzi = z[:, None] - z[None, :] + n - 1
    nv = l * m * n
    P = np.zeros((3 * nv, 3 * nv), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            P[a * nv:(a + 1) * nv, b * nv:(b + 1) * nv] = -dx ** 3 * C2[operator.comp_index(a, b)][dzi, dyi, dxi]
    P += ati * np.eye(3 * nv)
    inv = circulant.precond2_blocks(l, m, n, dx, k, ati)
    rng = np.random.default_rng(5)
    v = random_field((3, n, m, l), rng)
    Pv = (P @ v.reshape(-1)).reshape(v.shape)
    assert np.allclose(circulant.precond2_apply(Pv, inv), v, rtol=1e-11, atol=1e-11)


# Strang's circulant (named in Section 3 as the alternative to eq. 13).

def _strang_1d(t):
    return circulant.strang_axis(t[:, None], 0)[:, 0]


def test_strang_keeps_the_central_band():
    # C[i, j] = T[i, j] wherever |i - j| < L/2, checked on the dense matrices
    rng = np.random.default_rng(11)
    for L in (1, 2, 5, 6, 8):
        t = random_field(2 * L - 1, rng)
        T = circulant.toeplitz_dense(t)
        C = circulant.circulant_dense(_strang_1d(t))
        i, j = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
        band = 2 * np.abs(i - j) < L
        assert np.array_equal(C[band], T[band])
        if L % 2 == 0:  # the tie at |i - j| = L/2: mean of the two diagonals
            d = L // 2
            assert np.isclose(C[d, 0], 0.5 * (T[d, 0] + T[0, d]), rtol=1e-15)


def test_strang_fixed_point_and_parity():
    rng = np.random.default_rng(12)
    L = 8
    c = random_field(L, rng)
    t = np.array([c[o % L] for o in range(-(L - 1), L)])
    assert np.allclose(_strang_1d(t), c, rtol=1e-15, atol=0)
    # an odd Toeplitz symbol (t_{-o} = -t_o, as the xy/xz/yz blocks along an
    # odd axis) gives an odd circulant: c_{L-p} = -c_p, c_0 = c_{L/2} = 0
    h = random_field(L, rng)
    h[0] = 0
    t_odd = np.array([np.sign(o) * h[abs(o)] for o in range(-(L - 1), L)])
    s = _strang_1d(t_odd)
    assert s[0] == 0 and s[L // 2] == 0
    assert np.allclose(s[1:], -s[1:][::-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("comp", [0, 1, 2, 5])
def test_multilevel_strang_keeps_the_central_band(comp):
    # dense 3-level circulant from the closed form equals the BTTB block on
    # every pair whose x, y and z offsets all lie inside the central bands
    l, m, n, dx, k = 4, 5, 6, 0.3, 1.7
    T = circulant.bttb_block_dense(l, m, n, dx, k, comp)
    C3 = circulant.multilevel_circulant(l, m, n, dx, k, (True, True, True), "strang")[comp]
    z, y, x = np.meshgrid(np.arange(n), np.arange(m), np.arange(l), indexing="ij")
    x, y, z = x.reshape(-1), y.reshape(-1), z.reshape(-1)
    ox, oy, oz = x[:, None] - x[None, :], y[:, None] - y[None, :], z[:, None] - z[None, :]
    C = C3[oz % n, oy % m, ox % l]
    band = (2 * np.abs(ox) < l) & (2 * np.abs(oy) < m) & (2 * np.abs(oz) < n)
    assert np.allclose(C[band], T[band], rtol=1e-13, atol=1e-13 * np.abs(T).max())
    assert band.sum() > 0 and (~band).sum() > 0


@pytest.mark.parametrize("axis", ["x", "y"])
def test_precond2_other_toeplitz_axis_inverts_direct_construction(axis):
    # 2-level preconditioner with the Toeplitz level on x (y): assembled
    # directly as a dense matrix from the Chan circulant of the other two
    # levels, independently of the relabelling the oracle applies it with.
    from oracle.problem import Problem
    l, m, n, dx, k = 3, 4, 2, 0.5, 1.4
    levels = (False, True, True) if axis == "x" else (True, False, True)
    C2 = circulant.multilevel_circulant(l, m, n, dx, k, levels)
    z, y, x = np.meshgrid(np.arange(n), np.arange(m), np.arange(l), indexing="ij")
    x, y, z = x.reshape(-1), y.reshape(-1), z.reshape(-1)
    ox, oy, oz = x[:, None] - x[None, :], y[:, None] - y[None, :], z[:, None] - z[None, :]
    ix = ox + l - 1 if axis == "x" else ox % l
    iy = oy + m - 1 if axis == "y" else oy % m
    iz = oz % n
    mat = np.ones((n, m, l), dtype=np.uint8)
    prob = Problem(mat=mat, dx=dx, k=k, eps=[1.7 + 0.1j], d=np.array([0, 0, 1.0]),
                   e=np.array([1.0, 0, 0]))
    ati = prob.alpha_tilde_inv
    nv = l * m * n
    P = np.zeros((3 * nv, 3 * nv), dtype=np.complex128)
    for a in range(3):
        for b in range(3):
            P[a * nv:(a + 1) * nv, b * nv:(b + 1) * nv] = -dx ** 3 * C2[operator.comp_index(a, b)][iz, iy, ix]
    P += ati * np.eye(3 * nv)
    v = random_field((3, n, m, l), np.random.default_rng(9))
    Pv = (P @ v.reshape(-1)).reshape(v.shape)
    got = prob.precond2(restrict=False, axis=axis)(Pv)
    assert np.allclose(got, v, rtol=1e-11, atol=1e-11)
    # and it differs from the z-Toeplitz form (a different approximation)
    assert not np.allclose(prob.precond2(restrict=False)(Pv), v, rtol=1e-6, atol=1e-6)
