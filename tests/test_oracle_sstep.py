"""Pins of the oracle's s-step (Newton basis) GMRES: Leja ordering on point
sets whose order is known in closed form, the block Hessenberg formula
against the Arnoldi relation and against Arnoldi itself, and solutions and
iteration counts against direct solves and GMRES(m)."""
import numpy as np
import pytest

from dda_inputs import hex_prism_mask, random_field
from oracle import krylov, sstep
from oracle.problem import Problem


def test_leja_roots_of_unity_is_bit_reversal():
    # Leja points of the n-th roots of unity taken from 1 are the roots in
    # bit-reversed order (van der Corput sequence)
    z = np.exp(2j * np.pi * np.arange(8) / 8)
    assert sstep.leja_order(z, 8) == [0, 4, 2, 6, 1, 5, 3, 7]
    z16 = np.exp(2j * np.pi * np.arange(16) / 16)
    bitrev = [int(f"{k:04b}"[::-1], 2) for k in range(16)]
    order = sstep.leja_order(z16, 16)
    # ties may pick either of two mirror images; the product property is exact
    assert order[:4] == bitrev[:4]
    assert sorted(order) == list(range(16))


def test_leja_on_a_line_worked_by_hand():
    # first: largest modulus 2; then farthest from 2: -1; then the maximiser
    # of |z-2||z+1| among {-0.5, 0, 0.5, 1}: 0.5 (2.25); then -0.5 (1.25);
    # then 1 (1.5 against 0.5 for 0); then 0
    pts = [-1.0, -0.5, 0.0, 0.5, 1.0, 2.0]
    order = sstep.leja_order(pts, 6)
    assert [pts[i] for i in order] == [2.0, -1.0, 0.5, -0.5, 1.0, 0.0]
    assert sstep.leja_order(pts, 2) == order[:2]


def _random_op(n, seed, shift=4.0):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * shift + random_field((n, n), rng) / np.sqrt(n)
    return A, random_field(n, rng)


def _cycle(op, v0, m, s, theta):
    """One s-step cycle without Givens: (V, Hraw)."""
    V = np.zeros((m + 1, v0.size), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    V[0] = v0 / np.linalg.norm(v0)
    for j in range(0, m, s):
        W = sstep.newton_block(op, V[j], theta[:s])
        Qn, C, R = sstep.orthogonalise_block(V[:j + 1], W)
        H[:j + s + 1, j:j + s] = sstep.block_hessenberg(H, j, C, R, theta[:s])
        V[j + 1:j + s + 1] = Qn
    return V, H


@pytest.mark.parametrize("s", [1, 3, 4])
def test_block_hessenberg_satisfies_the_arnoldi_relation(s):
    n, m = 60, 12
    A, b = _random_op(n, 3)
    op = lambda v: A @ v
    theta = np.linalg.eigvals(A)[:s] * 0.9
    V, H = _cycle(op, b, m, s, theta)
    # A V_m = V_{m+1} H, V orthonormal, H upper Hessenberg, subdiagonal > 0
    lhs = A @ V[:m].T
    rhs = V.T @ H
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(lhs)
    assert np.linalg.norm(V.conj() @ V.T - np.eye(m + 1)) <= 1e-11
    assert np.all(np.tril(H, -2) == 0)
    sub = np.diag(H, -1)
    assert np.all(np.abs(sub.imag) <= 1e-12 * np.abs(sub)) and np.all(sub.real > 0)


def test_block_hessenberg_equals_arnoldi():
    # the Arnoldi factorisation with positive subdiagonal is unique: the
    # Newton blocks give the basis and the Hessenberg matrix of MGS Arnoldi
    n, m, s = 50, 10, 5
    A, b = _random_op(n, 4)
    op = lambda v: A @ v
    theta = np.array([4.2, 3.9 + 0.1j, 4.0 - 0.2j, 3.7, 4.4])
    V, H = _cycle(op, b, m, s, theta)
    Va = np.zeros_like(V)
    Ha = np.zeros_like(H)
    Va[0] = b / np.linalg.norm(b)
    for j in range(m):
        w = op(Va[j])
        for i in range(j + 1):
            Ha[i, j] = np.vdot(Va[i], w)
            w = w - Ha[i, j] * Va[i]
        Ha[j + 1, j] = np.linalg.norm(w)
        Va[j + 1] = w / Ha[j + 1, j]
    assert np.abs(H - Ha).max() <= 1e-10 * np.abs(Ha).max()
    assert np.abs(V - Va).max() <= 1e-10


@pytest.mark.parametrize("s", [1, 2, 5])
def test_sstep_solves_random_system(s):
    A, b = _random_op(40, 7)
    Minv = np.linalg.inv(np.diag(np.diag(A)))
    x, info = sstep.sstep_gmres(lambda v: A @ v, b, tol=1e-12, restart=10, maxiter=500,
                                precond=lambda v: Minv @ v, s=s)
    assert info["converged"]
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10
    assert info["shifts"] is not None and info["shifts"].size == s


def test_sstep_iterations_equal_gmres_on_dda_prism():
    l = m = n = 8
    dx, k = 2.0 / 8, 2.5
    mat = hex_prism_mask(l, m, n, dx, 1.0, 2.0)
    p = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=np.array([0, 0, 1.0]),
                e=np.array([1.0, 0, 0]))
    xd = p.solve_direct()
    Ghat = p.kernel_spectrum()
    mv = lambda v: p.matvec(v, Ghat)
    for pre in (None, p.precond3()):
        for restart in (6, 10):
            xg, ig = krylov.gmres(mv, p.rhs(), tol=1e-10, restart=restart, precond=pre)
            for s in (2, 3, 5):
                xs, info = sstep.sstep_gmres(mv, p.rhs(), tol=1e-10, restart=restart,
                                             precond=pre, s=s)
                assert info["converged"]
                assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) < 1e-8
                # the same iterates as GMRES(m): equal counts up to rounding
                assert abs(info["iters"] - ig["iters"]) <= 1, (restart, s)
                # products come in whole blocks: at most s - 1 extra per cycle
                assert ig["iters"] - 1 <= info["matvecs"] <= info["iters"] + (s - 1) * info["restarts"]


def test_ritz_shifts_take_the_leading_block():
    # a diagonal Hessenberg matrix: its leading 4s x 4s block has the
    # eigenvalues 1..20 (s = 5); Leja order from 20: 1, then the tie
    # |z - 20||z - 1| = 90 at 10 and 11 goes to 10 (first in order)
    H = np.zeros((31, 30), dtype=np.complex128)
    H[np.arange(30), np.arange(30)] = np.arange(1, 31)
    theta = sstep.ritz_shifts(H, 30, 5)
    assert np.allclose(theta[:3], [20, 1, 10])
    assert np.allclose(sstep.ritz_shifts(H, 3, 5), [3, 1, 2, 0, 0])
