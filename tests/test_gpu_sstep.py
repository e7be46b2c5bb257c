"""s-step GMRES (solve method 2) on the GPU: the Ritz-shift kernel against
numpy's eigenvalues and the Leja definition, whole solves against the
oracle's FP64 system, GMRES(m) on the same plan and the oracle's s-step
restatement, the graph-driven loop against the host-driven one, and the
option checks."""
import numpy as np
import pytest
import torch

from dda_inputs import prism_case
from gpu_util import dda_module, to_dev
from oracle import sstep as osstep
from oracle.problem import from_case


@pytest.mark.gpu
def test_ritz_shifts_are_leja_ordered_eigenvalues():
    dda = dda_module()
    rng = np.random.default_rng(5)
    m, s = 30, 5
    jl = [30, 12, 7, 3]
    H = np.zeros((len(jl), m, m + 1), dtype=np.complex128)  # row j = column j
    for r in range(len(jl)):
        A = np.triu(rng.standard_normal((m + 1, m)) + 1j * rng.standard_normal((m + 1, m)), -1)
        A[np.arange(1, m + 1), np.arange(m)] = np.abs(A[np.arange(1, m + 1), np.arange(m)])
        A[np.arange(m), np.arange(m)] += 3.0 * (r + 1)
        H[r] = A.T
    theta = dda.ritz_shifts(torch.from_numpy(H).cuda(),
                            torch.tensor(jl, dtype=torch.int32, device="cuda"), s).cpu().numpy()
    for r, j in enumerate(jl):
        k = min(j, 4 * s)
        ev = np.linalg.eigvals(H[r].T[:k, :k])
        scale = np.abs(ev).max()
        got = theta[r, :min(s, k)]
        # every shift is an eigenvalue of the leading block (the kernel
        # iterates in FP32), each at most once
        idx = [int(np.argmin(np.abs(ev - z))) for z in got]
        assert max(np.abs(ev[idx] - got)) <= 2e-5 * scale, r
        assert len(set(idx)) == len(idx)
        assert np.all(theta[r, min(s, k):] == 0)
        # Leja: the first of largest modulus, each next maximising the product
        # of distances to those taken (up to FP32 rounding)
        assert abs(got[0]) >= np.abs(ev).max() * (1 - 1e-4)
        for t in range(1, len(got)):
            left = [q for q in range(k) if q not in idx[:t]]
            prod = lambda q: np.prod(np.abs(ev[q] - ev[idx[:t]]))
            assert prod(idx[t]) >= max(prod(q) for q in left) * (1 - 1e-3), (r, t)
        # the oracle's shifts for the same matrix (its reading of the same steps)
        want = osstep.ritz_shifts(H[r].T, j, s)
        assert np.abs(want[:len(got)] - got).max() <= 2e-5 * scale, r


@pytest.fixture(scope="module")
def setup16():
    dda = dda_module()
    d2 = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    e2 = np.cross(d2, [0.0, 0.0, 1.0]) / np.linalg.norm(np.cross(d2, [0.0, 0.0, 1.0]))
    case = prism_case(16, 5.0, 1.31, 1.0, dirs=[[0.0, 0.0, 1.0], d2], pols=[[1.0, 0.0, 0.0], e2])
    prob = from_case(case)
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k, max_rhs=2,
                    krylov_m=50, precond2=True, sstep=5)
    plan.set_incidence(case.dirs, case.pols)
    plan.precond_build()
    plan.precond2_build()
    return dda, case, prob, plan


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("pc", [3, 0, 2])
def test_sstep_solve_matches_gmres_and_oracle(setup16, prec, pc):
    dda, case, prob, plan = setup16
    inner = dict(inner_prec=dda.C64, inner_tol=1e-4) if prec == "c64" else dict(inner_prec=dda.C128)
    kw = dict(tol=1e-6, restart=20, max_iters=1000, precond=pc, **inner)
    g = plan.solve(method=0, **kw)
    s = plan.solve(method=2, **kw)
    assert s.converged == [True, True] and s.status == 0
    assert max(s.rel_resid) <= 1e-6
    # the oracle's FP64 system, first incidence
    x = s.x[0].cpu().numpy()
    res = np.linalg.norm(prob.rhs() - prob.matvec(x)) / np.linalg.norm(prob.rhs())
    assert res <= 1e-6
    if prec == "c128":
        # the same GMRES(m) iterates: iteration counts equal up to rounding
        for a, b in zip(s.iters, g.iters):
            assert abs(a - b) <= 2, (s.iters, g.iters)
        if pc == 3:
            Ghat = prob.kernel_spectrum()
            _, info = osstep.sstep_gmres(lambda v: prob.matvec(v, Ghat), prob.rhs(), tol=1e-6,
                                         restart=20, precond=prob.precond3(), s=5)
            assert abs(s.iters[0] - info["iters"]) <= 3, (s.iters, info["iters"])
    else:
        for a, b in zip(s.iters, g.iters):
            assert a <= 1.2 * b + 5, (s.iters, g.iters)
    # cross sections of the two solvers agree to the solve tolerance
    cs, cg = plan.cross_sections(s.x), plan.cross_sections(g.x)
    assert np.abs(np.asarray(cs) - np.asarray(cg)).max() <= 1e-5 * np.abs(np.asarray(cg)).max()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_sstep_graph_equals_host_loop(setup16, prec):
    dda, case, prob, plan = setup16
    inner = dict(inner_prec=dda.C64, inner_tol=1e-4) if prec == "c64" else dict(inner_prec=dda.C128)
    kw = dict(tol=1e-6, restart=20, max_iters=1000, precond=3, method=2, **inner)
    plan.set_schedule(graph=False)
    host = plan.solve(history=4096, **kw)
    plan.set_schedule(graph=True)
    dev = plan.solve(history=4096, **kw)
    assert not host.graph and dev.graph
    assert dev.iters == host.iters and dev.cycles == host.cycles
    assert torch.equal(dev.x, host.x)
    for r in range(2):
        h = dev.history[r]
        assert len(h) == dev.iters[r] + 1 and h[0] == 1.0 and h[-1] == dev.rel_resid[r]
        assert np.array_equal(h, host.history[r])
    # a time limit stops the s-step solve too, and the plan stays usable
    t = plan.solve(timeout_ms=1e-6, raise_on_error=False, **kw)
    assert t.status == 9 and t.converged == [False, False]
    assert plan.solve(**kw).converged == [True, True]


@pytest.mark.gpu
def test_sstep_option_checks(setup16):
    dda, case, prob, plan = setup16
    with pytest.raises(dda.DDAError, match="multiple of sstep"):
        plan.solve(method=2, restart=22, precond=3)
    other = dda.Plan(plan.mat, case.eps, case.dx, case.k, max_rhs=2, krylov_m=20)
    other.set_incidence(case.dirs, case.pols)
    with pytest.raises(dda.DDAError, match="sstep"):
        other.solve(method=2, restart=20, precond=0)
