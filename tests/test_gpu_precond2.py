"""The paper's 2-level circulant preconditioner (Section 3, eqs. 17-19; the
block inversion of Section 3.1) on the GPU vs the oracle: apply parity,
solves, error paths.

The GPU inverts the 3n x 3n frequency blocks in complex64 and multiplies with
FP32 accumulation, so the tolerance is derived from the blocks' condition
number kappa (computed from the oracle's blocks): a backward-stable inverse
and an N-term product, N = 3n, with rounding errors that add up like a random
walk, give a relative error of order kappa * sqrt(N) * 2^-24 (a factor 4 of
headroom); the complex64 FFTs add about 1e-6.
"""
import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask, prism_case, random_field
from gpu_util import dda_module, rel_err, to_dev
from oracle import circulant
from oracle.problem import Problem, from_case

# (l, m, n): the block product streams the blocks through shared memory for
# even 3n <= 512 (one or two rows per thread), multiplies straight from global
# memory otherwise (n = 1, n = 256); unequal edges, thin boxes.
BOXES = [(4, 4, 4), (8, 4, 2), (16, 16, 16), (32, 16, 8), (2, 32, 16), (16, 8, 1),
         (2, 4, 128), (2, 4, 256)]
EPS32 = 2.0 ** -24


def _incidences():
    d1 = np.array([0.0, 0.0, 1.0]); e1 = np.array([1.0, 0.0, 0.0])
    d2 = np.array([0.3, -0.5, 0.8]); d2 /= np.linalg.norm(d2)
    e2 = np.cross(d2, [0, 0, 1.0]); e2 /= np.linalg.norm(e2)
    return [d1, d2], [e1, e2]


def _tolerance(prob):
    l, m, n = prob.dims
    binv = circulant.precond2_blocks(l, m, n, prob.dx, prob.k, prob.alpha_tilde_inv)
    kappa = max(np.linalg.cond(b) for b in binv.reshape(-1, 3 * n, 3 * n))
    return 2e-6 + 4 * kappa * np.sqrt(3 * n) * EPS32


@pytest.mark.gpu
@pytest.mark.parametrize("box", BOXES)
@pytest.mark.parametrize("full", [False, True])
def test_precond2_apply_parity(box, full):
    dda = dda_module()
    l, m, n = box
    rng = np.random.default_rng(300 + sum(box))
    if full:  # every voxel in the scatterer: restricted == unrestricted form
        mat = np.ones((n, m, l), dtype=np.uint8)
    else:
        mat = hex_prism_mask(l, m, n, 2.0 / max(l, m), 1.0, 2.0)
        if mat.sum() == 0:
            mat[0, 0, 0] = 1
    dx, k = 2.0 / max(l, m), 2.2
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2, precond2=True)
    plan.set_incidence(dirs, pols)
    plan.precond2_build()
    v = random_field((2, 3, n, m, l), rng)
    # one set of blocks per incidence batch: alpha_tilde of the first RHS
    prob = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[0], e=pols[0])
    apply = prob.precond2(restrict=not full)
    want = np.stack([apply(v[r]) for r in range(2)])
    tol = _tolerance(prob)
    z128 = plan.precond2_apply(to_dev(v)).cpu().numpy()
    assert rel_err(z128, want) < tol
    z64 = plan.precond2_apply(to_dev(v, torch.complex64)).cpu().numpy()
    assert rel_err(z64, want) < tol
    # in place (v and z the same buffer)
    vd = to_dev(v)
    plan.precond2_apply(vd, out=vd)
    assert rel_err(vd.cpu().numpy(), want) < tol
    # a single right-hand side (four vectors per block instead of eight)
    z1 = plan.precond2_apply(to_dev(v[:1], torch.complex64)).cpu().numpy()
    assert rel_err(z1, want[:1]) < tol


@pytest.mark.gpu
def test_precond2_apply_three_rhs():
    """Three right-hand sides: twelve mirrored vectors per block, two passes."""
    dda = dda_module()
    l, m, n = 8, 8, 4
    mat = hex_prism_mask(l, m, n, 0.25, 0.8, 1.0)
    dx, k = 0.25, 2.5
    dirs, pols = _incidences()
    dirs, pols = dirs + [np.array([1.0, 0, 0])], pols + [np.array([0, 0, 1.0])]
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=3, precond2=True)
    plan.set_incidence(dirs, pols)
    plan.precond2_build()
    v = random_field((3, 3, n, m, l), np.random.default_rng(11))
    prob = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[0], e=pols[0])
    apply = prob.precond2()
    want = np.stack([apply(v[r]) for r in range(3)])
    tol = _tolerance(prob)
    for dt in (torch.complex128, torch.complex64):
        assert rel_err(plan.precond2_apply(to_dev(v, dt)).cpu().numpy(), want) < tol


@pytest.mark.gpu
def test_precond2_inverts_the_two_level_operator():
    """P2^{-1} applied to P2 x gives x back (unrestricted, full box): checks the
    blocks against the dense 2-level matrix the oracle assembles independently
    of the block inverse."""
    dda = dda_module()
    l, m, n = 8, 4, 4
    mat = np.ones((n, m, l), dtype=np.uint8)
    dx, k = 0.25, 2.0
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.5 + 0.1j], dx, k, max_rhs=1, precond2=True)
    plan.set_incidence(dirs[:1], pols[:1])
    plan.precond2_build()
    prob = Problem(mat=mat, dx=dx, k=k, eps=[1.5 + 0.1j], d=dirs[0], e=pols[0])
    binv = circulant.precond2_blocks(l, m, n, dx, k, prob.alpha_tilde_inv)
    x = random_field((3, n, m, l), np.random.default_rng(7))
    # P2 x through the forward blocks (inverse of the oracle's inverse)
    blocks = np.linalg.inv(binv)
    X = np.fft.fftn(x, axes=(2, 3))
    Xb = np.moveaxis(X, (2, 3), (0, 1)).reshape(m, l, 3 * n)
    Yb = np.einsum("yxij,yxj->yxi", blocks, Xb)
    y = np.fft.ifftn(np.moveaxis(Yb.reshape(m, l, 3, n), (0, 1), (2, 3)), axes=(2, 3))
    got = plan.precond2_apply(to_dev(y[None])).cpu().numpy()[0]
    assert rel_err(got, x) < _tolerance(prob)


@pytest.fixture(scope="module")
def case16():
    dda = dda_module()
    case = prism_case(16, 5.0, 1.31, 1.0)
    prob = from_case(case)
    xd = prob.solve_direct()
    plan = dda.Plan(to_dev(case.mask(), torch.uint8), case.eps, case.dx, case.k, max_rhs=2,
                    krylov_m=50, precond2=True)
    plan.set_incidence(case.dirs, case.pols)
    plan.precond_build()
    plan.precond2_build()
    return dda, case, prob, xd, plan


@pytest.mark.gpu
@pytest.mark.parametrize("inner", ["c128", "c64"])
def test_precond2_solve_matches_direct(case16, inner):
    dda, case, prob, xd, plan = case16
    inner_prec = dda.C128 if inner == "c128" else dda.C64
    res = plan.solve(tol=1e-9, restart=50, precond=2, inner_prec=inner_prec, inner_tol=1e-4)
    x = res.x[0].cpu().numpy()
    assert res.converged[0]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6
    # the oracle's GMRES(50) with the same preconditioner (FP64 blocks)
    _, info = prob.solve_gmres("2", tol=1e-6, restart=50)
    res6 = plan.solve(tol=1e-6, restart=50, precond=2, inner_prec=dda.C128)
    assert abs(res6.iters[0] - info["iters"]) <= 2
    # Section 3.1: the 2-level form is the stronger preconditioner
    res3 = plan.solve(tol=1e-6, restart=50, precond=3, inner_prec=dda.C128)
    assert res6.iters[0] <= res3.iters[0]


@pytest.mark.gpu
def test_precond2_bicgstab(case16):
    dda, case, prob, xd, plan = case16
    res = plan.solve(tol=1e-8, max_iters=500, precond=2, inner_prec=dda.C128,
                     method=dda.BICGSTAB)
    x = res.x[0].cpu().numpy()
    assert res.converged[0]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-6


@pytest.mark.gpu
def test_precond2_error_paths():
    dda = dda_module()
    mat = np.ones((4, 4, 4), dtype=np.uint8)
    dirs, pols = _incidences()
    plain = dda.Plan(to_dev(mat, torch.uint8), [1.7], 0.3, 2.0, max_rhs=1, krylov_m=10)
    plain.set_incidence(dirs[:1], pols[:1])
    with pytest.raises(dda.DDAError, match="precond2"):
        plain.precond2_build()
    v = to_dev(random_field((1, 3, 4, 4, 4), np.random.default_rng(1)))
    with pytest.raises(dda.DDAError, match="DDA_ERR_NO_PRECOND"):
        plain.precond2_apply(v)
    with pytest.raises(dda.DDAError, match="DDA_ERR_NO_PRECOND"):
        plain.solve(tol=1e-6, restart=10, precond=2)
    p2 = dda.Plan(to_dev(mat, torch.uint8), [1.7], 0.3, 2.0, max_rhs=1, precond2=True)
    with pytest.raises(dda.DDAError, match="incidence"):
        p2.precond2_build()


@pytest.mark.gpu
@pytest.mark.parametrize("box", [(4, 4, 4), (16, 8, 1), (32, 16, 8)])
def test_precond2_apply_parity_strang(box):
    """2-level preconditioner with Strang's circulant on x and y."""
    dda = dda_module()
    l, m, n = box
    rng = np.random.default_rng(600 + sum(box))
    mat = hex_prism_mask(l, m, n, 2.0 / max(l, m), 1.0, 2.0)
    if mat.sum() == 0:
        mat[0, 0, 0] = 1
    dx, k = 2.0 / max(l, m), 2.2
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2, precond2=True,
                    circulant="strang")
    plan.set_incidence(dirs, pols)
    plan.precond2_build()
    v = random_field((2, 3, n, m, l), rng)
    prob = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[0], e=pols[0])
    apply = prob.precond2(kind="strang")
    want = np.stack([apply(v[r]) for r in range(2)])
    l_, m_, n_ = prob.dims
    binv = circulant.precond2_blocks(l_, m_, n_, dx, k, prob.alpha_tilde_inv, "strang")
    kappa = max(np.linalg.cond(b) for b in binv.reshape(-1, 3 * n, 3 * n))
    tol = 2e-6 + 4 * kappa * np.sqrt(3 * n) * EPS32
    assert rel_err(plan.precond2_apply(to_dev(v)).cpu().numpy(), want) < tol


@pytest.mark.gpu
@pytest.mark.parametrize("axis", ["x", "y"])
@pytest.mark.parametrize("box", [(4, 8, 16), (16, 4, 2), (8, 8, 8)])
def test_precond2_apply_parity_other_toeplitz_axis(axis, box):
    """2-level preconditioner with x or y as the Toeplitz level (the box
    relabelled so that level becomes z)."""
    dda = dda_module()
    l, m, n = box
    rng = np.random.default_rng(700 + sum(box))
    mat = hex_prism_mask(l, m, n, 2.0 / max(l, m), 1.0, 2.0)
    if mat.sum() == 0:
        mat[0, 0, 0] = 1
    dx, k = 2.0 / max(l, m), 2.2
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2, precond2=axis)
    plan.set_incidence(dirs, pols)
    plan.precond2_build()
    v = random_field((2, 3, n, m, l), rng)
    prob = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[0], e=pols[0])
    apply = prob.precond2(axis=axis)
    want = np.stack([apply(v[r]) for r in range(2)])
    fl, fm, fn = circulant.toeplitz_frame_dims(l, m, n, axis)
    binv = circulant.precond2_blocks(fl, fm, fn, dx, k, prob.alpha_tilde_inv)
    kappa = max(np.linalg.cond(b) for b in binv.reshape(-1, 3 * fn, 3 * fn))
    tol = 2e-6 + 4 * kappa * np.sqrt(3 * fn) * EPS32
    assert rel_err(plan.precond2_apply(to_dev(v)).cpu().numpy(), want) < tol
    assert rel_err(plan.precond2_apply(to_dev(v, torch.complex64)).cpu().numpy(), want) < tol
    # a solve with it reaches the direct solution
    plan2 = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2, krylov_m=50,
                     precond2=axis)
    plan2.set_incidence(dirs, pols)
    plan2.precond2_build()
    res = plan2.solve(tol=1e-9, restart=50, precond=2, inner_prec=dda.C64, inner_tol=1e-4)
    assert all(res.converged)
