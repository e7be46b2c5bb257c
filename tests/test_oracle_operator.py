"""Pins of the oracle's operator: Algorithm 1, dense assembly, FFT matvec."""
import numpy as np
import pytest

from dda_inputs import hex_prism_mask, pad_box, random_field, voxel_centres
from oracle import operator, physics
from oracle.problem import Problem


def _random_mask(shape, rng, frac=0.6):
    return (rng.random(shape) < frac).astype(np.uint8)


def test_alg1_tensor_entries():
    l, m, n, dx, k = 3, 4, 5, 0.4, 1.9
    G = operator.alg1_tensor(l, m, n, dx, k)
    assert G.shape == (6, n, m, l)
    assert np.all(G[:, 0, 0, 0] == 0)
    g = physics.green_tensor(np.array([2 * dx, 3 * dx, 1 * dx]), k)
    for c, (a, b) in enumerate(operator.COMPONENTS):
        assert G[c, 1, 3, 2] == g[a, b]


def test_circulant_generator_wrap_and_offsets():
    l, m, n, dx, k = 3, 2, 4, 0.5, 1.1
    gen = operator.circulant_generator(l, m, n, dx, k)
    assert gen.shape == (6, 2 * n, 2 * m, 2 * l)
    assert np.all(gen[:, :, :, l] == 0) and np.all(gen[:, :, m, :] == 0) and np.all(gen[:, n] == 0)
    g = physics.green_tensor(np.array([-1 * dx, 1 * dx, -3 * dx]), k)
    # offset (-1, 1, -3) sits at index (2l-1, 1, 2n-3)
    for c, (a, b) in enumerate(operator.COMPONENTS):
        assert np.isclose(gen[c, 2 * n - 3, 1, 2 * l - 1], g[a, b], rtol=1e-15)


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 3, 6), (7, 6, 5), (8, 8, 8)])
def test_fft_matvec_equals_dense(dims):
    l, m, n = dims
    rng = np.random.default_rng(sum(dims))
    mat = _random_mask((n, m, l), rng)
    mat[0, 0, 0] = 1
    k, dx = 1.3, 0.35
    ainv = operator.alpha_inv_box(mat, [physics.alpha_ldr(1.7 + 0.1j, k, dx, 0.2)])
    c = random_field((3, n, m, l), rng)
    y = operator.fft_matvec(c, mat, ainv, 5.0 + 1.0j, k, dx)
    A = operator.dense_matrix(mat, ainv, k, dx)
    want = operator.ice_to_box(A @ operator.box_to_ice(c, mat), mat)
    ice = mat > 0
    err = np.abs(y - want)[:, ice].max() / np.abs(want).max()
    assert err < 1e-12
    # air rows: alpha_tilde^{-1} c
    assert np.allclose(y[:, ~ice], (5.0 + 1.0j) * c[:, ~ice], rtol=1e-15, atol=0)


def test_dense_matrix_complex_symmetric():
    rng = np.random.default_rng(1)
    mat = _random_mask((4, 5, 6), rng)
    k, dx = 2.0, 0.3
    ainv = operator.alpha_inv_box(mat, [physics.alpha_ldr(2.0, k, dx, 0.0)])
    A = operator.dense_matrix(mat, ainv, k, dx)
    assert np.allclose(A, A.T, rtol=0, atol=1e-13 * np.abs(A).max())
    assert not np.allclose(A, A.conj().T)


def test_fft_matvec_bilinear_symmetry():
    # u^T (A v) = (A u)^T v with the unconjugated product (A = A^T)
    rng = np.random.default_rng(2)
    l, m, n = 6, 5, 4
    mat = _random_mask((n, m, l), rng)
    k, dx = 1.1, 0.5
    ainv = operator.alpha_inv_box(mat, [physics.alpha_ldr(1.9, k, dx, 0.1)])
    u = random_field((3, n, m, l), rng)
    v = random_field((3, n, m, l), rng)
    Av = operator.fft_matvec(v, mat, ainv, 3.0, k, dx)
    Au = operator.fft_matvec(u, mat, ainv, 3.0, k, dx)
    lhs = np.sum(u * Av)
    rhs = np.sum(Au * v)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_air_padding_leaves_solution_unchanged():
    # Padding the box with air (even margins keep the centre) changes
    # neither the scatterer's unknowns nor the incident field on them.
    l = m = n = 6
    dx, k = 2.0 / 6, 2.0
    mat = hex_prism_mask(l, m, n, dx, 1.0, 2.0)
    big = pad_box(mat, l + 4, m + 2, n + 6)
    d = np.array([0.3, -0.4, 0.866]); d /= np.linalg.norm(d)
    e = np.cross(d, [0, 0, 1.0]); e /= np.linalg.norm(e)
    p0 = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=d, e=e)
    p1 = Problem(mat=big, dx=dx, k=k, eps=[1.31 ** 2], d=d, e=e)
    x0, i0 = p0.solve_gmres("none", tol=1e-12, restart=200)
    x1, i1 = p1.solve_gmres("none", tol=1e-12, restart=200)
    v0 = operator.box_to_ice(x0, mat)
    v1 = operator.box_to_ice(x1, big)
    assert np.linalg.norm(v1 - v0) / np.linalg.norm(v0) < 1e-10
    # and the direct solve agrees with GMRES
    xd = p0.solve_direct()
    assert np.linalg.norm(operator.box_to_ice(xd, mat) - v0) / np.linalg.norm(v0) < 1e-10


def test_matvec_rows_equal_dense_rows():
    rng = np.random.default_rng(21)
    l, m, n = 6, 5, 4
    mat = _random_mask((n, m, l), rng)
    k, dx = 1.4, 0.3
    ainv = operator.alpha_inv_box(mat, [physics.alpha_ldr(1.9 + 0.1j, k, dx, 0.3)])
    c = random_field((3, n, m, l), rng)
    full = operator.fft_matvec(c, mat, ainv, 4.0 - 1.0j, k, dx)
    rows = list(range(0, l * m * n, 7))
    got = operator.matvec_rows(c, mat, ainv, 4.0 - 1.0j, k, dx, rows)
    want = full.reshape(3, -1)[:, rows].T
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(full).max())
