"""Adjoint gradient dC_ext/d(eps) per voxel on the GPU vs the oracle (and finite differences)."""
import numpy as np
import pytest
import torch

from dda_inputs import config2_cases, hex_prism_mask, prism_case
from gpu_util import dda_module, rel_err, to_dev
from oracle import adjoint, operator
from oracle.problem import Problem, from_case


def _dirs():
    d = np.array([0.3, -0.2, 0.93]); d /= np.linalg.norm(d)
    e = np.cross(d, [0, 0, 1.0]); e /= np.linalg.norm(e)
    return d, e


def _oracle_solutions(prob):
    A = operator.dense_matrix(prob.mat, prob.alpha_inv_vox, prob.k, prob.dx)
    c = operator.ice_to_box(np.linalg.solve(A, operator.box_to_ice(prob.rhs(), prob.mat)), prob.mat)
    lam = operator.ice_to_box(np.linalg.solve(A, operator.box_to_ice(adjoint.adjoint_rhs(prob), prob.mat)),
                              prob.mat)
    return c, lam


@pytest.mark.gpu
def test_adjoint_rhs_and_gradient_arithmetic():
    dda = dda_module()
    l = m = n = 8
    dx, k = 0.25, 2.2
    mat = hex_prism_mask(l, m, n, dx, 1.0, 2.0)
    d, e = _dirs()
    eps = (1.31 + 0.01j) ** 2
    prob = Problem(mat=mat, dx=dx, k=k, eps=[eps], d=d, e=e)
    plan = dda.Plan(to_dev(mat, torch.uint8), [eps], dx, k, max_rhs=1, krylov_m=30)
    plan.set_incidence([d], [e])
    assert rel_err(plan.adjoint_rhs().cpu().numpy()[0], adjoint.adjoint_rhs(prob)) < 1e-13
    c, lam = _oracle_solutions(prob)
    g = plan.ext_gradient_from(to_dev(c)[None], to_dev(lam)[None]).cpu().numpy()[0]
    assert rel_err(g, adjoint.ext_gradient(prob, c, lam)) < 1e-12


@pytest.mark.gpu
def test_gpu_gradient_matches_finite_differences():
    dda = dda_module()
    l = m = n = 8  # prism of ~140 voxels in an air-padded 8^3 box
    dx, k = 0.25, 2.2
    mat = hex_prism_mask(l, m, n, dx, 0.75, 1.5)
    d, e = _dirs()
    eps = (1.31 + 0.02j) ** 2
    plan = dda.Plan(to_dev(mat, torch.uint8), [eps], dx, k, max_rhs=1, krylov_m=40)
    plan.set_incidence([d], [e])
    plan.precond_build()
    _, _, grad = plan.ext_gradient(tol=1e-12, restart=40, precond=3, inner_prec=dda.C128)
    grad = grad.cpu().numpy()[0]
    rng = np.random.default_rng(5)
    ice = np.argwhere(mat > 0)
    h = 1e-6
    for t in rng.choice(len(ice), 4, replace=False):
        z, y, x = ice[t]
        for comp, step in ((0, h), (1, 1j * h)):
            vals = []
            for sgn in (+1, -1):
                mat2 = mat.copy()
                mat2[z, y, x] = 2
                p2 = Problem(mat=mat2, dx=dx, k=k, eps=[eps, eps + sgn * step], d=d, e=e)
                vals.append(adjoint.c_ext_of(p2, p2.solve_direct()))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(grad[comp, z, y, x] - fd) <= 1e-4 * abs(fd) + 1e-6 * np.abs(grad).max()


@pytest.mark.gpu
def test_gradient_64cube_every_voxel():
    # The 64^3 differentiation workload (x = 20, m = 1.31 + 0.01i): solve and
    # adjoint solve on the GPU (complex64 cycles, FP64 refinement), gradient
    # for every voxel.  Checked against the oracle's gradient arithmetic on
    # the same fields and by the oracle's residuals of both solves.
    dda = dda_module()
    case = prism_case(64, 20.0, 1.31 + 0.01j, 1.0)
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k, max_rhs=1,
                    krylov_m=50)
    plan.set_incidence(case.dirs, case.pols)
    plan.precond_build()
    c, lam, grad = plan.ext_gradient(tol=1e-8, restart=50, precond=3, inner_prec=dda.C64,
                                     inner_tol=1e-4)
    prob = from_case(case, 0)
    cn, ln = c.cpu().numpy()[0], lam.cpu().numpy()[0]
    b, bl = prob.rhs(), adjoint.adjoint_rhs(prob)
    G = prob.kernel_spectrum()
    assert np.linalg.norm(b - prob.matvec(cn, G)) / np.linalg.norm(b) <= 1e-8
    assert np.linalg.norm(bl - prob.matvec(ln, G)) / np.linalg.norm(bl) <= 1e-8
    assert rel_err(grad.cpu().numpy()[0], adjoint.ext_gradient(prob, cn, ln)) < 1e-12
