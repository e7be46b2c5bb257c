"""The solve loop as one CUDA graph launch (device-side restart, convergence,
iteration-cap and time-limit decisions) against the host-driven loop and the
oracle; the residual history and the time limit."""
import numpy as np
import pytest
import torch

from dda_inputs import prism_case
from gpu_util import dda_module, to_dev
from oracle.problem import from_case


@pytest.fixture(scope="module")
def setup16():
    dda = dda_module()
    d2 = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    e2 = np.cross(d2, [0.0, 0.0, 1.0]) / np.linalg.norm(np.cross(d2, [0.0, 0.0, 1.0]))
    case = prism_case(16, 5.0, 1.31, 1.0, dirs=[[0.0, 0.0, 1.0], d2], pols=[[1.0, 0.0, 0.0], e2])
    prob = from_case(case)
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k, max_rhs=2,
                    krylov_m=50, precond2=True)
    plan.set_incidence(case.dirs, case.pols)
    plan.precond_build()
    plan.precond2_build()
    return dda, case, prob, plan


SOLVERS = [dict(precond=3, method=0), dict(precond=0, method=0), dict(precond=2, method=0),
           dict(precond=3, method=1), dict(precond=2, method=1)]


@pytest.mark.gpu
@pytest.mark.late(2)
@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("kw", SOLVERS, ids=lambda k: f"p{k['precond']}m{k['method']}")
def test_graph_solve_equals_host_loop(setup16, prec, kw):
    dda, case, prob, plan = setup16
    inner = dict(inner_prec=dda.C64, inner_tol=1e-4) if prec == "c64" else dict(inner_prec=dda.C128)
    opts = dict(tol=1e-6, restart=20, max_iters=1000, **inner, **kw)
    plan.set_schedule(graph=False)
    host = plan.solve(**opts)
    plan.set_schedule(graph=True)
    first = plan.solve(**opts)     # captures the graph
    x_first = first.x.clone()
    del first.x
    again = plan.solve(**opts)     # reuses it if x lands at the same address, else recaptures
    assert not host.graph and again.graph
    for g, x in ((first, x_first), (again, again.x)):
        assert g.graph
        assert g.iters == host.iters and g.cycles == host.cycles
        assert g.converged == host.converged == [True, True]
        assert torch.equal(x, host.x)
        assert g.rel_resid == host.rel_resid
    # the solution satisfies the oracle's FP64 system (first incidence)
    x = x_first[0].cpu().numpy()
    res = np.linalg.norm(prob.rhs() - prob.matvec(x)) / np.linalg.norm(prob.rhs())
    assert res <= 1e-6


@pytest.mark.gpu
@pytest.mark.late(2)
def test_residual_history(setup16):
    dda, case, prob, plan = setup16
    for graph in (True, False):
        plan.set_schedule(graph=graph)
        res = plan.solve(tol=1e-6, restart=20, precond=3, inner_prec=dda.C64, inner_tol=1e-4,
                         history=4096)
        for r in range(2):
            h = res.history[r]
            assert len(h) == res.iters[r] + 1
            assert h[0] == 1.0                         # x0 = 0: ||b - A 0|| / ||b||
            assert h[-1] == res.rel_resid[r] <= 1e-6   # the final FP64 residual
            assert np.all(np.isfinite(h)) and np.all(h > 0)
            # GMRES's estimate never grows within a cycle: rises only where a
            # restart replaced the estimate by the true FP64 residual
            rises = int(np.sum(h[1:] > h[:-1] * (1 + 1e-12)))
            assert rises <= res.cycles[r]
        short = plan.solve(tol=1e-6, restart=20, precond=3, inner_prec=dda.C64, inner_tol=1e-4,
                           history=5)
        assert [len(h) for h in short.history] == [5, 5]
        assert np.array_equal(short.history[0], res.history[0][:5])
    plan.set_schedule(graph=True)


@pytest.mark.gpu
@pytest.mark.late(2)
@pytest.mark.parametrize("graph", [True, False])
@pytest.mark.parametrize("method", [0, 1])
def test_time_limit_stops_the_solve(setup16, graph, method):
    """A 1 ns limit stops every right-hand side at its first check with
    DDA_ERR_TIMEOUT (no GPU wait is involved: the limit is compared with the
    device clock after each iteration and at each restart); the plan and the
    context stay usable: the next solve without a limit converges."""
    dda, case, prob, plan = setup16
    plan.set_schedule(graph=graph)
    kw = dict(tol=1e-6, restart=20, precond=3, inner_prec=dda.C64, inner_tol=1e-4, method=method)
    res = plan.solve(timeout_ms=1e-6, raise_on_error=False, history=64, **kw)
    assert res.status == 9  # DDA_ERR_TIMEOUT
    assert res.converged == [False, False]
    assert max(res.iters) <= 1
    ok = plan.solve(**kw)
    assert ok.converged == [True, True] and ok.status == 0
    plan.set_schedule(graph=True)


@pytest.mark.gpu
@pytest.mark.late(2)
def test_graph_solve_counts_its_kernels(setup16):
    """The graph counts the kernels it runs on the device; the host-driven
    loop counts its launches.  The host loop runs at most one extra step per
    cycle (it launches a step before it sees the last one's decision) and one
    scale kernel less per cycle, so the two counts agree within that."""
    dda, case, prob, plan = setup16
    kw = dict(tol=1e-6, restart=20, precond=3, inner_prec=dda.C64, inner_tol=1e-4)
    counts = {}
    for graph in (False, True):
        plan.set_schedule(graph=graph)
        plan.solve(**kw)  # capture outside the count
        n0 = dda.launch_count()
        res = plan.solve(**kw)
        counts[graph] = dda.launch_count() - n0
    per_step = 5 + 5 + 4 + 2  # preconditioner, matvec, two Gram-Schmidt passes, Givens, scale
    cycles = max(res.cycles)
    assert counts[True] > per_step * max(res.iters)
    assert abs(counts[True] - counts[False]) <= (per_step + 1) * (cycles + 1)
    plan.set_schedule(graph=True)
