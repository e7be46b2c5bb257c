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
