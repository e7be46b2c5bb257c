"""The GPU solver on the paper's own experiment (Section 4): a thin hexagonal
plate, plane wave along +x polarised along z, x = 10, with the 2-level
preconditioner.  The GPU needs power-of-two box edges, so the plate's
39 x 34 x 2 box (mu = 1.2, L/a = 0.1) is grown with air to 64 x 64 x 2; the
oracle solves the same padded box, and the GPU must agree on the iteration
count and the solution."""
import math

import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask
from gpu_util import dda_module, to_dev
from oracle.problem import Problem


@pytest.mark.gpu
@pytest.mark.parametrize("mu, n", [(1.2, 2), (1.8, 4)])
def test_paper_plate_two_level_solve(mu, n):
    dda = dda_module()
    x, a = 10.0, 1.0
    k = x / a
    dx = 2 * math.pi / (10 * mu * k)
    l = m = 64
    mat = hex_prism_mask(l, m, n, dx, a, n * dx)
    d, e = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    prob = Problem(mat=mat, dx=dx, k=k, eps=[mu ** 2], d=d, e=e)
    x_ref, info = prob.solve_gmres("2", tol=1e-10, restart=50, maxiter=500)
    assert info["converged"]
    plan = dda.Plan(to_dev(mat, torch.uint8), [mu ** 2], dx, k, max_rhs=1, krylov_m=50,
                    precond2=True)
    plan.set_incidence([d], [e])
    plan.precond2_build()
    res = plan.solve(tol=1e-10, restart=50, precond=2, inner_prec=dda.C128)
    assert res.converged[0]
    xg = res.x[0].cpu().numpy()
    assert np.linalg.norm(xg - x_ref) / np.linalg.norm(x_ref) < 1e-8
    _, info6 = prob.solve_gmres("2", tol=1e-5, restart=50, maxiter=500)
    res6 = plan.solve(tol=1e-5, restart=50, precond=2, inner_prec=dda.C128)
    assert abs(res6.iters[0] - info6["iters"]) <= 2
    # and with complex64 cycles inside FP64 refinement
    res64 = plan.solve(tol=1e-5, restart=50, precond=2, inner_prec=dda.C64, inner_tol=1e-3)
    assert res64.converged[0]


@pytest.mark.gpu
@pytest.mark.late(5)
def test_paper_plate_x20_two_level_solve():
    # the x = 20 row of Table 3 for mu = 1.2 (L/a = 0.1: 77 x 67 x 4 plate box),
    # grown with air to 128 x 128 x 4; GPU against the oracle on that box
    dda = dda_module()
    mu, n, x, a = 1.2, 4, 20.0, 1.0
    k = x / a
    dx = 2 * math.pi / (10 * mu * k)
    l = m = 128
    mat = hex_prism_mask(l, m, n, dx, a, n * dx)
    d, e = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.0, 1.0])
    prob = Problem(mat=mat, dx=dx, k=k, eps=[mu ** 2], d=d, e=e)
    x_ref, info = prob.solve_gmres("2", tol=1e-10, restart=50, maxiter=500)
    assert info["converged"]
    plan = dda.Plan(to_dev(mat, torch.uint8), [mu ** 2], dx, k, max_rhs=1, krylov_m=50,
                    precond2=True)
    plan.set_incidence([d], [e])
    plan.precond2_build()
    res = plan.solve(tol=1e-10, restart=50, precond=2, inner_prec=dda.C128)
    assert res.converged[0]
    xg = res.x[0].cpu().numpy()
    assert np.linalg.norm(xg - x_ref) / np.linalg.norm(x_ref) < 1e-8
    _, info5 = prob.solve_gmres("2", tol=1e-5, restart=50, maxiter=500)
    res5 = plan.solve(tol=1e-5, restart=50, precond=2, inner_prec=dda.C128)
    assert abs(res5.iters[0] - info5["iters"]) <= 2
