"""Many incident waves in one solve (the directions-by-polarisations batch of
an orientation average): 12 seeded directions x 2 polarisations = 24
right-hand sides of a 16^3 prism (x = 5, m = 1.31 + 0.01i) advance in lock
step through complex64 GMRES cycles with FP64 refinement; every one must reach
the tolerance and give the oracle's cross sections for its own incidence (the
LDR polarizability differs per wave through S)."""
import numpy as np
import pytest
import torch

from dda_inputs import polarisations, prism_case, random_direction
from gpu_util import dda_module, to_dev
from oracle.problem import Problem


@pytest.mark.gpu
@pytest.mark.late(2)
def test_24_waves_in_one_batch():
    dda = dda_module()
    case = prism_case(16, 5.0, 1.31 + 0.01j, 1.0)
    rng = np.random.default_rng(1)
    dirs, pols = [], []
    for _ in range(12):
        d = random_direction(rng)
        for e in polarisations(d):
            dirs.append(d)
            pols.append(e)
    mat = case.mask()
    plan = dda.Plan(to_dev(mat, torch.uint8), case.eps, case.dx, case.k, max_rhs=24, krylov_m=50)
    plan.set_incidence(dirs, pols)
    plan.precond_build()
    res = plan.solve(tol=1e-6, restart=50, precond=3, inner_prec=dda.C64, inner_tol=1e-4)
    assert all(res.converged) and max(res.rel_resid) <= 1e-6
    got = plan.cross_sections(res.x)
    for r in (0, 13, 23):
        prob = Problem(mat=mat, dx=case.dx, k=case.k, eps=list(case.eps), d=dirs[r], e=pols[r])
        want = np.array(prob.cross_sections(prob.solve_direct()))
        assert np.abs(got[r] - want).max() <= 1e-5 * np.abs(want).max(), r


@pytest.mark.gpu
@pytest.mark.late(2)
def test_rhs_chunks_give_the_same_results():
    """A plan whose FFT scratch holds rhs_chunk right-hand sides passes larger
    batches through the transforms in chunks: the matvec (both precisions),
    both preconditioners and a whole solve of 5 waves with chunks of 2 equal
    the unchunked plan's bit for bit (the per-line transforms are the same)."""
    dda = dda_module()
    case = prism_case(16, 5.0, 1.31 + 0.01j, 1.0)
    rng = np.random.default_rng(4)
    dirs, pols = [], []
    for _ in range(5):
        d = random_direction(rng)
        dirs.append(d)
        pols.append(polarisations(d)[0])
    mat = to_dev(case.mask(), torch.uint8)
    plans = []
    for chunk in (0, 2):
        pl = dda.Plan(mat, case.eps, case.dx, case.k, max_rhs=5, krylov_m=30, precond2=True,
                      rhs_chunk=chunk)
        pl.set_incidence(dirs, pols)
        pl.precond_build()
        pl.precond2_build()
        plans.append(pl)
    assert dda.workspace_size(16, 16, 16, case.dx, case.k, 1, 5, 30, rhs_chunk=2) < \
        dda.workspace_size(16, 16, 16, case.dx, case.k, 1, 5, 30)
    x = torch.randn((5, 3, 16, 16, 16), dtype=torch.complex128, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(9))
    for t in (x, x.to(torch.complex64)):
        assert torch.equal(plans[0].matvec(t), plans[1].matvec(t))
        assert torch.equal(plans[0].precond_apply(t), plans[1].precond_apply(t))
        assert torch.equal(plans[0].precond2_apply(t), plans[1].precond2_apply(t))
    res = [pl.solve(tol=1e-6, restart=30, precond=3, inner_prec=dda.C64, inner_tol=1e-4)
           for pl in plans]
    assert res[0].iters == res[1].iters and torch.equal(res[0].x, res[1].x)
    assert torch.equal(torch.as_tensor(plans[0].cross_sections(res[0].x)),
                       torch.as_tensor(plans[1].cross_sections(res[1].x)))


@pytest.mark.gpu
@pytest.mark.late(2)
def test_complex64_krylov_reservation():
    """krylov_c64: the basis and step vectors reserved in complex64 (half the
    memory); complex64 cycles give the same solution as on a plan reserving
    complex128, bit for bit, and complex128 cycles are refused."""
    dda = dda_module()
    case = prism_case(16, 5.0, 1.31 + 0.01j, 1.0)
    mat = to_dev(case.mask(), torch.uint8)
    assert dda.workspace_size(16, 16, 16, case.dx, case.k, 1, 1, 30, krylov_c64=True) < \
        dda.workspace_size(16, 16, 16, case.dx, case.k, 1, 1, 30)
    res = []
    for c64 in (False, True):
        pl = dda.Plan(mat, case.eps, case.dx, case.k, max_rhs=1, krylov_m=30, krylov_c64=c64)
        pl.set_incidence(case.dirs, case.pols)
        pl.precond_build()
        res.append(pl.solve(tol=1e-6, restart=30, precond=3, inner_prec=dda.C64, inner_tol=1e-4))
    assert res[0].iters == res[1].iters and torch.equal(res[0].x, res[1].x)
    with pytest.raises(dda.DDAError, match="krylov_c64"):
        pl.solve(tol=1e-6, restart=30, precond=3, inner_prec=dda.C128)
