"""Pins of the adjoint gradient: closed-form derivative and central finite differences."""
import numpy as np
import pytest

from dda_inputs import hex_prism_mask
from oracle import adjoint, physics
from oracle.problem import Problem


def test_dalpha_inv_matches_finite_difference():
    for eps in (1.31 ** 2, (1.6 + 0.1j) ** 2):
        for S in (0.0, 0.4):
            k, dx, h = 2.0, 0.3, 1e-6
            f = lambda e: 1.0 / physics.alpha_ldr(e, k, dx, S)
            fd = (f(eps + h) - f(eps - h)) / (2 * h)
            assert abs(adjoint.dalpha_inv_deps(eps, k, dx, S) - fd) < 1e-6 * abs(fd)


def _problem(eps_list, mat):
    d = np.array([0.3, -0.2, 0.93]); d /= np.linalg.norm(d)
    e = np.cross(d, [0, 0, 1.0]); e /= np.linalg.norm(e)
    return Problem(mat=mat, dx=0.25, k=2.2, eps=eps_list, d=d, e=e)


def test_adjoint_gradient_equals_central_differences():
    l = m = n = 6
    mat = hex_prism_mask(l, m, n, 0.25, 0.75, 1.5)
    eps = (1.31 + 0.02j) ** 2
    prob = _problem([eps], mat)
    c = prob.solve_direct()
    lam = prob_adj = None
    # adjoint solve with the same (complex-symmetric) matrix
    A_rhs = adjoint.adjoint_rhs(prob)
    from oracle import operator
    A = operator.dense_matrix(mat, prob.alpha_inv_vox, prob.k, prob.dx)
    lam = operator.ice_to_box(np.linalg.solve(A, operator.box_to_ice(A_rhs, mat)), mat)
    grad = adjoint.ext_gradient(prob, c, lam)
    rng = np.random.default_rng(3)
    ice = np.argwhere(mat > 0)
    h = 1e-6
    for t in rng.choice(len(ice), 5, replace=False):
        z, y, x = ice[t]
        for comp, step in ((0, h), (1, 1j * h)):
            vals = []
            for sgn in (+1, -1):
                mat2 = mat.copy()
                mat2[z, y, x] = 2
                p2 = _problem([eps, eps + sgn * step], mat2)
                vals.append(adjoint.c_ext_of(p2, p2.solve_direct()))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(grad[comp, z, y, x] - fd) <= 1e-5 * np.abs(grad).max()
    assert np.all(grad[:, mat == 0] == 0)
