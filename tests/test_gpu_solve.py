"""Solver parity: GMRES on the GPU vs the oracle (16^3 prism, x = 5, m = 1.31)."""
import numpy as np
import pytest
import torch

from dda_inputs import prism_case, hex_prism_mask
from gpu_util import dda_module, rel_err, to_dev
from oracle import observables
from oracle.problem import Problem, from_case


@pytest.fixture(scope="module")
def case16():
    dda = dda_module()
    case = prism_case(16, 5.0, 1.31, 1.0)
    prob = from_case(case)
    xd = prob.solve_direct()
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k, max_rhs=2,
                    krylov_m=50)
    plan.set_incidence(case.dirs, case.pols)
    plan.precond_build()
    return dda, case, prob, xd, plan


def _true_resid(prob, x):
    r = prob.rhs() - prob.matvec(x)
    return np.linalg.norm(r) / np.linalg.norm(prob.rhs())


@pytest.mark.gpu
@pytest.mark.parametrize("precond", [0, 3])
def test_c128_gmres_matches_direct_solve(case16, precond):
    dda, case, prob, xd, plan = case16
    res = plan.solve(tol=1e-6, restart=50, precond=precond, inner_prec=dda.C128)
    x = res.x[0].cpu().numpy()
    assert res.converged[0] and res.rel_resid[0] <= 1e-6
    assert _true_resid(prob, x) <= 1e-6
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-4
    # same algorithm as the oracle's GMRES(50) up to Gram-Schmidt rounding
    _, info = prob.solve_gmres("3" if precond else "none", tol=1e-6, restart=50)
    assert abs(res.iters[0] - info["iters"]) <= 2


@pytest.mark.gpu
def test_tight_tolerance_reaches_direct_solution(case16):
    dda, case, prob, xd, plan = case16
    res = plan.solve(tol=1e-11, restart=50, precond=3, inner_prec=dda.C128)
    x = res.x[0].cpu().numpy()
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("precond", [0, 3])
def test_mixed_precision_refinement(case16, precond):
    dda, case, prob, xd, plan = case16
    res = plan.solve(tol=1e-6, restart=50, precond=precond, inner_prec=dda.C64, inner_tol=1e-4)
    x = res.x[0].cpu().numpy()
    assert res.converged[0]
    assert _true_resid(prob, x) <= 1e-6
    cext_o = prob.cross_sections(xd)[0]
    cext = plan.cross_sections(res.x)[0, 0]
    assert abs(cext - cext_o) / abs(cext_o) <= 1e-5


@pytest.mark.gpu
def test_cross_sections_parity_and_optical_theorem(case16):
    dda, case, prob, xd, plan = case16
    got = plan.cross_sections(to_dev(xd)[None])[0]
    cext, cabs, csca = prob.cross_sections(xd, pairs=True)
    assert abs(got[0] - cext) <= 1e-10 * abs(cext)
    assert abs(got[2] - csca) <= 1e-9 * abs(csca)
    assert abs(got[1] - cabs) <= 1e-9 * abs(cext)  # real m: C_abs ~ 0
    assert abs(got[0] - got[1] - got[2]) <= 1e-8 * got[0]


@pytest.mark.gpu
def test_absorbing_cross_sections_parity():
    dda = dda_module()
    case = prism_case(8, 2.5, 1.31 + 0.05j, 1.0)
    prob = from_case(case)
    xd = prob.solve_direct()
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k)
    plan.set_incidence(case.dirs, case.pols)
    got = plan.cross_sections(to_dev(xd)[None])[0]
    want = prob.cross_sections(xd, pairs=True)
    assert rel_err(np.array(got), np.array(want)) < 1e-9


@pytest.mark.gpu
def test_batched_rhs_equal_single_solves(case16):
    dda, case, prob, xd, plan = case16
    d2 = np.array([0.6, 0.0, 0.8]); e2 = np.array([0.0, 1.0, 0.0])
    plan.set_incidence([case.dirs[0], d2], [case.pols[0], e2])
    both = plan.solve(tol=1e-8, restart=50, precond=3, inner_prec=dda.C128)
    plan.set_incidence([d2], [e2])
    one = plan.solve(tol=1e-8, restart=50, precond=3, inner_prec=dda.C128)
    p2 = Problem(mat=prob.mat, dx=prob.dx, k=prob.k, eps=prob.eps, d=d2, e=e2)
    x2 = one.x[0].cpu().numpy()
    assert _true_resid(p2, x2) <= 1e-8
    assert np.linalg.norm(both.x[1].cpu().numpy() - x2) / np.linalg.norm(x2) < 1e-7
    assert both.iters[1] == one.iters[0]
    plan.set_incidence(case.dirs, case.pols)


@pytest.mark.gpu
def test_solver_edge_cases(case16):
    dda, case, prob, xd, plan = case16
    l, m, n = case.dims
    zero_b = torch.zeros((1, 3, n, m, l), dtype=torch.complex128, device="cuda")
    res = plan.solve(b=zero_b, tol=1e-6, precond=3)
    assert res.converged[0] and res.iters[0] == 0 and float(res.x.abs().max()) == 0.0
    # the iteration cap is honoured and reported
    res = plan.solve(tol=1e-12, max_iters=5, restart=50, precond=0, raise_on_error=False)
    assert dda.STATUS[res.status] == "DDA_ERR_NOT_CONVERGED" and res.iters[0] == 5
    # a NaN in the right-hand side is reported, not iterated on
    bad = plan.incident_field(1)
    bad[0, 0, 0, 0, 0] = float("nan")
    res = plan.solve(b=bad, tol=1e-6, precond=0, raise_on_error=False)
    assert dda.STATUS[res.status] == "DDA_ERR_NAN"
    # restart larger than the plan reserved
    with pytest.raises(dda.DDAError):
        plan.solve(tol=1e-6, restart=51)


@pytest.mark.gpu
@pytest.mark.late(1)
def test_resume_from_a_stopped_solve(case16):
    # checkpoint and resume: a solve stopped by the iteration cap keeps its
    # last iterate (and reports its true residual); a solve started from it
    # finishes the job
    dda, case, prob, xd, plan = case16
    part = plan.solve(tol=1e-8, max_iters=10, restart=50, precond=0, inner_prec=dda.C128,
                      raise_on_error=False)
    assert dda.STATUS[part.status] == "DDA_ERR_NOT_CONVERGED" and part.iters[0] == 10
    r_part = _true_resid(prob, part.x[0].cpu().numpy())
    assert r_part < 0.05 and part.rel_resid[0] == pytest.approx(r_part, rel=1e-6)
    rest = plan.solve(x0=part.x, tol=1e-8, restart=50, precond=0, inner_prec=dda.C128)
    assert all(rest.converged)
    x = rest.x[0].cpu().numpy()
    assert _true_resid(prob, x) <= 1.1e-8
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6


@pytest.mark.gpu
def test_precond_required_before_use():
    dda = dda_module()
    mat = hex_prism_mask(8, 8, 8, 0.25, 1.0, 2.0)
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.7161], 0.25, 2.5, krylov_m=10)
    plan.set_incidence([[0, 0, 1.0]], [[1.0, 0, 0]])
    with pytest.raises(dda.DDAError) as e:
        plan.solve(tol=1e-6, restart=10, precond=3)
    assert "DDA_ERR_NO_PRECOND" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("precond", [0, 3])
def test_bicgstab_matches_direct_and_oracle(case16, precond):
    dda, case, prob, xd, plan = case16
    from oracle import krylov
    res = plan.solve(tol=1e-6, restart=200, precond=precond, inner_prec=dda.C128,
                     method=dda.BICGSTAB)
    x = res.x[0].cpu().numpy()
    assert res.converged[0] and _true_resid(prob, x) <= 1e-6
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-4
    G = prob.kernel_spectrum()
    _, info = krylov.bicgstab(lambda v: prob.matvec(v, G), prob.rhs(), tol=1e-6,
                              precond=prob.precond3() if precond else None)
    assert abs(res.iters[0] - info["iters"]) <= max(3, info["iters"] // 10)


@pytest.mark.gpu
def test_bicgstab_mixed_precision(case16):
    dda, case, prob, xd, plan = case16
    res = plan.solve(tol=1e-6, restart=30, precond=3, inner_prec=dda.C64, inner_tol=1e-4,
                     method=dda.BICGSTAB)
    x = res.x[0].cpu().numpy()
    assert res.converged[0] and _true_resid(prob, x) <= 1e-6
