"""Pins of the oracle's restarted GMRES against direct solves."""
import numpy as np
import pytest

from dda_inputs import random_field
from oracle import krylov, operator
from oracle.problem import Problem
from dda_inputs import hex_prism_mask


@pytest.mark.parametrize("side", ["right", "left"])
@pytest.mark.parametrize("restart", [5, 40])
def test_gmres_random_system(side, restart):
    rng = np.random.default_rng(7)
    n = 40
    A = np.eye(n) * 4 + random_field((n, n), rng) / np.sqrt(n)
    b = random_field(n, rng)
    Minv = np.linalg.inv(np.diag(np.diag(A)))
    x, info = krylov.gmres(lambda v: A @ v, b, tol=1e-12, restart=restart, maxiter=500,
                           precond=lambda v: Minv @ v, side=side)
    assert info["converged"]
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-10


def test_gmres_full_terminates_within_n():
    rng = np.random.default_rng(8)
    n = 12
    A = random_field((n, n), rng) + 3 * np.eye(n)
    b = random_field(n, rng)
    x, info = krylov.gmres(lambda v: A @ v, b, tol=1e-13, restart=n, maxiter=n)
    assert info["iters"] <= n and info["converged"]
    # full GMRES residual estimates never increase
    h = np.array(info["history"])
    assert np.all(np.diff(h) <= 1e-14)


def test_gmres_residual_estimate_matches_true_residual():
    rng = np.random.default_rng(9)
    n = 30
    A = random_field((n, n), rng) + 6 * np.eye(n)
    b = random_field(n, rng)
    x, info = krylov.gmres(lambda v: A @ v, b, tol=1e-8, restart=n, maxiter=n)
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert abs(true - info["history"][-1]) < 1e-10


def test_gmres_dda_prism_matches_direct():
    l = m = n = 8
    dx, k = 2.0 / 8, 2.5
    mat = hex_prism_mask(l, m, n, dx, 1.0, 2.0)
    p = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=np.array([0, 0, 1.0]), e=np.array([1.0, 0, 0]))
    xd = p.solve_direct()
    for pre in ("none", "3", "2"):
        x, info = p.solve_gmres(pre, tol=1e-10, restart=30)
        assert info["converged"]
        err = np.linalg.norm(x - xd) / np.linalg.norm(xd)
        assert err < 1e-8, (pre, err)
        r = p.rhs() - p.matvec(x)
        assert np.linalg.norm(r) / np.linalg.norm(p.rhs()) <= 1e-10


def test_bicgstab_random_and_dda():
    rng = np.random.default_rng(17)
    n = 40
    A = np.eye(n) * 4 + random_field((n, n), rng) / np.sqrt(n)
    b = random_field(n, rng)
    Minv = np.linalg.inv(np.diag(np.diag(A)))
    x, info = krylov.bicgstab(lambda v: A @ v, b, tol=1e-12, precond=lambda v: Minv @ v)
    assert info["converged"]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) / np.linalg.norm(b) < 1e-10
    l = m = n3 = 8
    dx, k = 2.0 / 8, 2.5
    mat = hex_prism_mask(l, m, n3, dx, 1.0, 2.0)
    p = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=np.array([0, 0, 1.0]), e=np.array([1.0, 0, 0]))
    xd = p.solve_direct()
    G = p.kernel_spectrum()
    for M in (None, p.precond3()):
        x, info = krylov.bicgstab(lambda v: p.matvec(v, G), p.rhs(), tol=1e-10, precond=M)
        assert info["converged"]
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
