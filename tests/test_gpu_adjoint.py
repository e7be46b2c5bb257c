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


def _relabel_per_voxel(mat, eps_vox):
    """The oracle's form of a per-voxel permittivity: one material per
    scatterer voxel (at most 255 of them)."""
    idx = np.argwhere(mat > 0)
    assert len(idx) <= 255
    relab = np.zeros_like(mat)
    for q, (z, y, x) in enumerate(idx):
        relab[z, y, x] = q + 1
    return relab, [complex(eps_vox[z, y, x]) for z, y, x in idx]


@pytest.mark.gpu
@pytest.mark.late(3)
def test_voxel_eps_operator_solve_and_gradient_vs_oracle():
    """dda_set_voxel_eps: the matvec, a solve's cross sections and the
    adjoint gradient with a different permittivity in every voxel, against the
    oracle with one material per voxel."""
    dda = dda_module()
    l, m, n = 8, 8, 4
    dx, k = 0.3, 2.0
    mat = hex_prism_mask(l, m, n, dx, 1.15, 1.2)
    rng = np.random.default_rng(21)
    eps_vox = ((1.4 + 0.03j) + 0.25 * rng.standard_normal(mat.shape)
               + 0.03j * rng.random(mat.shape)) ** 2
    relab, eps_list = _relabel_per_voxel(mat, eps_vox)
    d, e = _dirs()
    prob = Problem(mat=relab, dx=dx, k=k, eps=eps_list, d=d, e=e)
    plan = dda.Plan(to_dev(mat, torch.uint8), [eps_list[0]], dx, k, max_rhs=1, krylov_m=40,
                    voxel_eps=to_dev(eps_vox))
    plan.set_incidence([d], [e])
    x = np.random.default_rng(3).standard_normal((1, 3, n, m, l)) * (1 + 0.5j)
    want = prob.matvec(x[0])
    assert rel_err(plan.matvec(to_dev(x)).cpu().numpy()[0], want) < 1e-10
    assert rel_err(plan.matvec(to_dev(x, torch.complex64)).cpu().numpy()[0], want) < 2e-5
    plan.precond_build()
    c_gpu, lam_gpu, g_gpu = plan.ext_gradient(tol=1e-12, restart=40, precond=3,
                                              inner_prec=dda.C128)
    c, lam = _oracle_solutions(prob)
    assert rel_err(c_gpu.cpu().numpy()[0], c) < 1e-9
    xs = plan.cross_sections(c_gpu)[0]
    cext, cabs, csca = prob.cross_sections(c, pairs=True)
    assert abs(xs[0] - cext) <= 1e-9 * abs(cext)
    assert abs(xs[1] - cabs) <= 1e-9 * abs(cext)
    assert abs(xs[2] - csca) <= 1e-9 * abs(cext)
    assert rel_err(g_gpu.cpu().numpy()[0], adjoint.ext_gradient(prob, c, lam)) < 1e-8
    # switching the table off restores the per-material operator
    plan.set_voxel_eps(None)
    prob1 = Problem(mat=mat, dx=dx, k=k, eps=[eps_list[0]], d=d, e=e)
    assert rel_err(plan.matvec(to_dev(x)).cpu().numpy()[0], prob1.matvec(x[0])) < 1e-10


@pytest.mark.gpu
@pytest.mark.late(4)
def test_voxel_gradient_64cube_vs_central_differences():
    """The 64^3 prism at x = 20, m = 1.31 + 0.01i: the adjoint gradient
    dC_ext/d eps for every voxel (dda.extinction with a permittivity per
    voxel) against central differences (step 1e-6) on 32 seeded scatterer
    voxels.  Each perturbed solution is x0 + delta with A(eps +- h) delta =
    b - A(eps +- h) x0 solved to 1e-10 relative to that right-hand side (the
    perturbed system solved from the unperturbed solution x0, which cancels
    out of the difference exactly); C_ext is linear in the field, so the
    difference quotient is C_ext(delta+ - delta-)/2h."""
    dda = dda_module()
    case = prism_case(64, 20.0, 1.31 + 0.01j, 1.0)
    mat = case.mask()
    n, m, l = mat.shape
    eps0 = complex(case.eps[0])
    d, e = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    mat_t = to_dev(mat, torch.uint8)
    eps = torch.full((n, m, l), eps0, dtype=torch.complex128, device="cuda", requires_grad=True)
    kw = dict(tol=1e-12, restart=50, precond=3, inner_prec=dda.C128, max_iters=3000)
    cext = dda.extinction(eps, mat_t, case.dx, case.k, [d], [e], **kw)
    cext.sum().backward()
    grad = eps.grad.cpu().numpy()
    assert np.all(grad[mat == 0] == 0)
    # finite differences with the library's own operator and solver
    ve = torch.full((n, m, l), eps0, dtype=torch.complex128, device="cuda")
    plan = dda.Plan(mat_t, [eps0], case.dx, case.k, max_rhs=1, krylov_m=50, voxel_eps=ve)
    plan.set_incidence([d], [e])
    plan.precond_build()
    x0 = plan.solve(**kw).x
    b = plan.incident_field(1)
    rng = np.random.default_rng(3)
    ice = np.argwhere(mat > 0)
    h = 1e-6
    got, fd = [], []
    for t in rng.choice(len(ice), 32, replace=False):
        z, y, x = ice[t]
        for unit in (1.0, 1j):
            deltas = []
            for sgn in (1.0, -1.0):
                vp = ve.clone()
                vp[z, y, x] += sgn * h * unit
                plan.set_voxel_eps(vp)
                rhs = b - plan.matvec(x0)
                deltas.append(plan.solve(b=rhs, tol=1e-10, restart=50, precond=3,
                                         inner_prec=dda.C128, max_iters=3000).x)
            dq = plan.cross_sections(deltas[0] - deltas[1])[0, 0] / (2 * h)
            fd.append(dq)
            g = grad[z, y, x]
            got.append(g.real if unit == 1.0 else g.imag)
        plan.set_voxel_eps(ve)
    got, fd = np.array(got), np.array(fd)
    assert np.abs(got - fd).max() <= 1e-4 * np.abs(fd).max()
    assert np.all(np.abs(got - fd) <= 1e-3 * np.abs(fd) + 1e-6 * np.abs(fd).max())
