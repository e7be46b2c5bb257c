"""Parity at the benchmark's sizes, in the benchmark's launch configuration.

64^3: whole matvecs against the oracle's FFT matvec, and solves of the
benchmark sweep against the oracle's own iteration counts
(tests/golden/config2_oracle_iters.txt, written by oracle/iteration_counts.py)
with the true residual evaluated by the oracle.  128^3: sampled rows against
direct summation.  256^3: the complex symmetry u^T A v = (A u)^T v, which holds
at any size.
"""
import os

import numpy as np
import pytest
import torch

from dda_inputs import config2_cases, prism_case, random_field
from gpu_util import dda_module, rel_err, to_dev
from oracle import operator
from oracle.problem import from_case

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "config2_oracle_iters.txt")


def _golden_iters():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out[(int(f[0]), int(f[1]), int(f[2]), round(float(f[3]), 4), round(float(f[4]), 4),
                 int(f[5]))] = int(f[6])
    return out


def _plan(dda, case, krylov_m=0):
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k,
                    max_rhs=case.nrhs, krylov_m=krylov_m)
    plan.set_incidence(case.dirs, case.pols)
    return plan


@pytest.mark.gpu
def test_matvec_64cube_whole_field():
    dda = dda_module()
    case = config2_cases()[4]  # 64^3, m = 1.31 + 0.05i, aspect 1, two polarisations
    plan = _plan(dda, case)
    rng = np.random.default_rng(64)
    x = random_field((2, 3) + case.mask().shape, rng)
    want = []
    for r in range(2):
        prob = from_case(case, r)
        want.append(prob.matvec(x[r]))
    want = np.stack(want)
    assert rel_err(plan.matvec(to_dev(x)).cpu().numpy(), want) < 1e-10
    assert rel_err(plan.matvec(to_dev(x, torch.complex64)).cpu().numpy(), want) < 2e-5


@pytest.mark.gpu
def test_matvec_128cube_sampled_rows():
    dda = dda_module()
    case = prism_case(128, 40.0, 1.31 + 0.01j, 1.0)  # the 128^3 precision workload
    plan = _plan(dda, case)
    prob = from_case(case, 0)
    rng = np.random.default_rng(128)
    x = random_field((1, 3) + case.mask().shape, rng)
    y128 = plan.matvec(to_dev(x)).cpu().numpy()[0]
    y64 = plan.matvec(to_dev(x, torch.complex64)).cpu().numpy()[0]
    mat = case.mask()
    ice = np.flatnonzero(mat.reshape(-1) > 0)
    air = np.flatnonzero(mat.reshape(-1) == 0)
    rows = list(rng.choice(ice, 10, replace=False)) + list(rng.choice(air, 2, replace=False))
    want = operator.matvec_rows(x[0], mat, prob.alpha_inv_vox, prob.alpha_tilde_inv, prob.k,
                                prob.dx, rows)
    scale = np.abs(want).max()
    for got, tol in ((y128, 1e-10), (y64, 2e-5)):
        g = got.reshape(3, -1)[:, rows].T
        assert np.abs(g - want).max() / scale < tol


@pytest.mark.gpu
def test_matvec_256cube_complex_symmetry():
    dda = dda_module()
    case = prism_case(256, 80.0, 1.31, 1.0)
    plan = _plan(dda, case)
    shape = (1, 3) + case.mask().shape
    g = torch.Generator(device="cuda").manual_seed(256)
    u = torch.randn(shape, dtype=torch.complex128, device="cuda", generator=g)
    v = torch.randn(shape, dtype=torch.complex128, device="cuda", generator=g)
    Av = plan.matvec(v)
    Au = plan.matvec(u)
    lhs = complex(torch.sum(u * Av))
    rhs = complex(torch.sum(Au * v))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    del Av, Au
    u32, v32 = u.to(torch.complex64), v.to(torch.complex64)
    lhs32 = complex(torch.sum(u32.to(torch.complex128) * plan.matvec(v32).to(torch.complex128)))
    rhs32 = complex(torch.sum(plan.matvec(u32).to(torch.complex128) * v32.to(torch.complex128)))
    assert abs(lhs32 - rhs32) < 1e-5 * abs(lhs32)


@pytest.mark.gpu
# the six converging systems of the 64^3 sweep: m = 1.31 (0-2) and
# m = 1.31 + 0.05i (3-5), aspects 0.5, 1, 2 (boxes 64x64x32, 64^3, 64x64x128)
@pytest.mark.parametrize("idx", [0, 1, 2, 3, 4, 5])
def test_solve_bench_configuration(idx):
    dda = dda_module()
    case = config2_cases()[idx]
    plan = _plan(dda, case, krylov_m=50)
    plan.precond_build()
    res = plan.solve(tol=1e-6, restart=50, precond=3, inner_prec=dda.C64, inner_tol=1e-4,
                     max_iters=2000, reorth_eta=0.1)
    golden = _golden_iters()
    eps = complex(case.eps[0])
    xs = res.x.cpu().numpy()
    for r in range(2):
        prob = from_case(case, r)
        b = prob.rhs()
        rel = np.linalg.norm(b - prob.matvec(xs[r])) / np.linalg.norm(b)
        assert res.converged[r] and rel <= 1e-6
        key = case.dims + (round(eps.real, 4), round(eps.imag, 4), r)
        assert abs(res.iters[r] - golden[key]) <= 2, (res.iters[r], golden[key])
    got = plan.cross_sections(res.x)
    for r in range(2):
        prob = from_case(case, r)
        want = np.array(prob.cross_sections(xs[r]))
        assert np.abs(got[r] - want).max() <= 1e-9 * abs(want[0])


def _twin_golden():
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "config3_twin32_oracle.txt")):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            vals[f[0]] = [float(v) for v in f[1:]]
    return vals


@pytest.mark.gpu
@pytest.mark.late(1)
def test_config3_twin_mixed_precision_vs_oracle():
    """The 32^3 twin of the 128^3 precision workload (x = 10, k dx = 0.625,
    m = 1.31 + 0.01i): complex64 GMRES cycles inside FP64 refinement to 1e-6,
    C_ext and C_sca against the oracle's FP64 solve (to 1e-12, stored by
    oracle/twin_values.py): relative error <= 1e-5."""
    dda = dda_module()
    case = prism_case(32, 10.0, 1.31 + 0.01j, 1.0)
    want = _twin_golden()
    assert int(want["box"][3]) == int((case.mask() > 0).sum())
    plan = _plan(dda, case, krylov_m=50)
    plan.precond_build()
    res = plan.solve(tol=1e-6, restart=50, precond=3, inner_prec=dda.C64, inner_tol=1e-4,
                     max_iters=2000, reorth_eta=0.1, nrhs=1)
    assert res.converged[0]
    got = plan.cross_sections(res.x)[0]
    for i, name in ((0, "c_ext"), (2, "c_sca")):
        assert abs(got[i] - want[name][0]) <= 1e-5 * abs(want[name][0]), (name, got[i], want[name])
