"""Boxes with even 7-smooth edges (mixed-radix transforms of radix 2, 4, 3, 5,
7): the 3-D FFT against numpy.fft, the matvec and both preconditioners
against the oracle, solves against the dense direct solve, and the 96^3
prism of the 128-wave batch in its own box against the same prism padded
with air to 128^3 (air padding leaves the solution unchanged)."""
import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask, prism_case, random_field
from gpu_util import dda_module, rel_err, to_dev
from oracle.problem import Problem, from_case
from test_gpu_operator import _incidences, _oracle_box_matvec, _two_material_box
from test_gpu_precond2 import _tolerance

# lengths l, m, n and their padded 2l, 2m, 2n cover the radices 3, 5, 7 alone
# and combined, one and several power-of-two stages (transforms of 12 = 4 x 3
# leave the last stage unpruned), edges of 2, ragged tiles
FFT_SHAPES = [(6, 10, 14), (24, 20, 12), (96, 30, 8), (2, 42, 28), (90, 2, 6), (40, 56, 70)]
BOXES = [(6, 10, 14), (24, 20, 12), (12, 36, 30), (10, 6, 48), (30, 28, 2), (96, 6, 6),
         (14, 16, 42)]


@pytest.mark.gpu
@pytest.mark.late(6)
@pytest.mark.parametrize("shape", FFT_SHAPES)
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_fft3d_mixed_radix_matches_numpy(shape, prec):
    dda = dda_module()
    l, m, n = shape
    mat = torch.ones((n, m, l), dtype=torch.uint8, device="cuda")
    plan = dda.Plan(mat, [2.0], 0.1, 1.0, precisions=dda.PLAN_C128 | dda.PLAN_C64)
    rng = np.random.default_rng(l * 7 + m * 3 + n)
    a = random_field((3, n, m, l), rng)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    tol = 1e-12 if prec == "c128" else 3e-6
    t = to_dev(a, dt)
    plan.fft3d(t)
    want = np.fft.fftn(a, axes=(1, 2, 3))
    assert rel_err(t.cpu().numpy(), want) < tol
    plan.fft3d(t, inverse=True)
    assert rel_err(t.cpu().numpy(), a) < tol


@pytest.mark.gpu
@pytest.mark.late(6)
@pytest.mark.parametrize("box", BOXES)
def test_matvec_parity_mixed_radix(box):
    dda = dda_module()
    l, m, n = box
    rng = np.random.default_rng(sum(box))
    mat = _two_material_box(l, m, n, rng)
    eps = [1.31 ** 2, (1.6 + 0.05j) ** 2]
    dx, k = 0.3, 1.7
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), eps, dx, k, max_rhs=2)
    plan.set_incidence(dirs, pols)
    x = random_field((2, 3, n, m, l), rng)
    want = np.stack([_oracle_box_matvec(mat, eps, dx, k, dirs[r], pols[r], x[r])[0]
                     for r in range(2)])
    assert rel_err(plan.matvec(to_dev(x)).cpu().numpy(), want) < 1e-10
    assert rel_err(plan.matvec(to_dev(x, torch.complex64)).cpu().numpy(), want) < 2e-5


@pytest.mark.gpu
@pytest.mark.late(6)
@pytest.mark.parametrize("box", BOXES)
def test_precond_apply_parity_mixed_radix(box):
    dda = dda_module()
    l, m, n = box
    rng = np.random.default_rng(100 + sum(box))
    mat = hex_prism_mask(l, m, n, 2.0 / max(l, m), 1.0, 2.0)
    if mat.sum() == 0:
        mat[0, 0, 0] = 1
    dx, k = 2.0 / max(l, m), 2.2
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2)
    plan.set_incidence(dirs, pols)
    plan.precond_build()
    v = random_field((2, 3, n, m, l), rng)
    want = np.stack([Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[r], e=pols[r])
                     .precond3()(v[r]) for r in range(2)])
    assert rel_err(plan.precond_apply(to_dev(v)).cpu().numpy(), want) < 1e-10
    assert rel_err(plan.precond_apply(to_dev(v, torch.complex64)).cpu().numpy(), want) < 2e-5


@pytest.mark.gpu
@pytest.mark.late(6)
@pytest.mark.parametrize("box", [(6, 10, 14), (24, 20, 12), (30, 12, 6)])
def test_precond2_apply_parity_mixed_radix(box):
    dda = dda_module()
    l, m, n = box
    rng = np.random.default_rng(300 + sum(box))
    mat = hex_prism_mask(l, m, n, 2.0 / max(l, m), 1.0, 2.0)
    if mat.sum() == 0:
        mat[0, 0, 0] = 1
    dx, k = 2.0 / max(l, m), 2.2
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2, precond2=True)
    plan.set_incidence(dirs, pols)
    plan.precond2_build()
    v = random_field((2, 3, n, m, l), rng)
    prob = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[0], e=pols[0])
    apply = prob.precond2()
    want = np.stack([apply(v[r]) for r in range(2)])
    tol = _tolerance(prob)
    assert rel_err(plan.precond2_apply(to_dev(v)).cpu().numpy(), want) < tol
    assert rel_err(plan.precond2_apply(to_dev(v, torch.complex64)).cpu().numpy(), want) < tol


@pytest.mark.gpu
@pytest.mark.late(6)
def test_solve_mixed_radix_box_matches_direct():
    """The 14^3 prism (k dx = 0.625, m = 1.31): GMRES(50) with the 3-level
    preconditioner in complex128 and in complex64 + FP64 refinement, against
    the oracle's dense direct solve and its GMRES iteration count."""
    dda = dda_module()
    case = prism_case(14, 14 * 0.3125, 1.31, 1.0)
    assert case.dims == (14, 14, 14)
    prob = from_case(case)
    xd = prob.solve_direct()
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k, max_rhs=1,
                    krylov_m=50)
    plan.set_incidence(case.dirs, case.pols)
    plan.precond_build()
    res = plan.solve(tol=1e-10, restart=50, precond=3, inner_prec=dda.C128)
    x = res.x[0].cpu().numpy()
    assert res.converged[0]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
    res6 = plan.solve(tol=1e-6, restart=50, precond=3, inner_prec=dda.C128)
    _, info = prob.solve_gmres("3", tol=1e-6, restart=50)
    assert abs(res6.iters[0] - info["iters"]) <= 2
    resm = plan.solve(tol=1e-6, restart=50, precond=3, inner_prec=dda.C64, inner_tol=1e-4)
    xm = resm.x[0].cpu().numpy()
    r = prob.rhs() - prob.matvec(xm)
    assert np.linalg.norm(r) / np.linalg.norm(prob.rhs()) <= 1e-6
    xs = plan.cross_sections(resm.x)[0]
    want = prob.cross_sections(xd)
    assert abs(xs[0] - want[0]) / abs(want[0]) < 1e-5  # C_ext after refinement
    # cross sections of the exact solution, on the GPU and in the oracle
    got = plan.cross_sections(to_dev(xd)[None])[0]
    for q in range(3):
        assert abs(got[q] - want[q]) <= 1e-9 * abs(want[0]), q


@pytest.mark.gpu
@pytest.mark.late(7)
def test_prism96_own_box_equals_air_padded_box():
    """The 96^3 prism of the many-wave batch (x = 30, m = 1.31, seeded
    direction, both polarisations) solved in its own 96^3 box (transform
    lengths 192 = 4 x 3 x 4 x 4 and 96) and in the 128^3 box that holds it:
    air padding leaves the solution on the scatterer unchanged, so C_ext,
    C_sca and the scatterer's field agree to the solves' residual 1e-6."""
    dda = dda_module()
    rng = np.random.default_rng(1)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    e1 = np.cross(d, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    out = {}
    for box in [(96, 96, 96), (128, 128, 128)]:
        case = prism_case(96, 30.0, 1.31, 1.0, dirs=[d, d], pols=[e1, e2])
        case.box = box
        plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k, max_rhs=2,
                        krylov_m=50)
        plan.set_incidence(case.dirs, case.pols)
        plan.precond_build()
        res = plan.solve(tol=1e-6, restart=50, precond=3, inner_prec=dda.C64, inner_tol=1e-4)
        assert all(res.converged), (box, res.iters, res.rel_resid)
        x = res.x.cpu().numpy()
        o = (box[0] - 96) // 2  # the prism's 96^3 block inside the box
        out[box] = (x[:, :, o:o + 96, o:o + 96, o:o + 96], plan.cross_sections(res.x),
                    case.mask())
        del plan
        torch.cuda.empty_cache()
    (xa, sa, ma), (xb, sb, mb) = out[(96, 96, 96)], out[(128, 128, 128)]
    o = 16
    assert np.array_equal(ma, mb[o:o + 96, o:o + 96, o:o + 96])
    assert rel_err(xa, xb) < 1e-4
    for r in range(2):
        for q in (0, 2):  # C_ext, C_sca
            assert abs(sa[r, q] - sb[r, q]) / abs(sb[r, q]) < 1e-5, (r, q, sa[r], sb[r])
