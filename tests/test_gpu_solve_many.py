"""dda_solve_many: several independent systems solved concurrently (one host
thread and one stream per plan) give exactly the results of the same solves
run one by one, on an uneven batch of prisms."""
import numpy as np
import pytest
import torch

from dda_inputs import prism_case
from gpu_util import dda_module, to_dev

CASES = [(16, 5.0, 1.31, 1.0), (16, 5.0, 1.31 + 0.05j, 0.5), (32, 8.0, 1.31, 1.0),
         (16, 5.0, 1.4, 2.0)]


def _plans(dda):
    plans = []
    for N, x, m, asp in CASES:
        case = prism_case(N, x, m, asp)
        plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k,
                        max_rhs=2, krylov_m=30)
        plan.set_incidence(case.dirs, case.pols)
        plan.precond_build()
        plans.append(plan)
    return plans


@pytest.mark.gpu
@pytest.mark.parametrize("method", ["gmres", "bicgstab"])
def test_solve_many_equals_single_solves(method):
    dda = dda_module()
    plans = _plans(dda)
    kw = dict(tol=1e-6, restart=30, precond=3, inner_prec=dda.C64, inner_tol=1e-4,
              method=dda.GMRES if method == "gmres" else dda.BICGSTAB)
    single = [p.solve(**kw) for p in plans]
    many = dda.solve_many(plans, **kw)
    torch.cuda.synchronize()
    for a, b in zip(single, many):
        assert a.iters == b.iters and a.converged == b.converged
        assert all(a.converged)
        assert torch.equal(a.x, b.x)


@pytest.mark.gpu
def test_solve_many_rejects_shared_plans_and_streams():
    dda = dda_module()
    plans = _plans(dda)[:2]
    with pytest.raises(dda.DDAError, match="appears twice"):
        dda.solve_many([plans[0], plans[0]])
    s = torch.cuda.Stream()
    with pytest.raises(dda.DDAError, match="share a stream"):
        dda.solve_many(plans, streams=[s, s])
    # a failing member (iteration cap) is reported with its index, the others still solve
    res = dda.solve_many(plans, max_iters=3, raise_on_error=False)
    assert res[0].status != 0
    assert not any(res[0].converged)
