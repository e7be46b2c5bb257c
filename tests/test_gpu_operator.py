"""K2-K7 parity: matvec and preconditioner apply of the CUDA path vs the oracle."""
import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask, random_field
from gpu_util import dda_module, rel_err, to_dev
from oracle import circulant, operator, physics
from oracle.problem import Problem

# (l, m, n): several FFT tiles per pass, ragged tails (lines not a multiple of
# the tile), unequal edges, a 1-voxel-thick box; n = 32 and 64 take the
# matvec's register-resident z pass (z transforms of length 64 and 128), with
# rows of the padded plane shorter and longer than its column tile; n = 128
# the all-shared-memory z pass of length 256.
BOXES = [(4, 4, 4), (8, 4, 2), (16, 16, 16), (32, 16, 8), (2, 32, 16), (16, 8, 1),
         (8, 4, 32), (4, 8, 64), (16, 8, 32), (4, 4, 128)]


def _two_material_box(l, m, n, rng):
    mat = (rng.random((n, m, l)) < 0.55).astype(np.uint8)
    mat[rng.random((n, m, l)) < 0.2] *= 2
    return mat


def _incidences():
    d1 = np.array([0.0, 0.0, 1.0]); e1 = np.array([1.0, 0.0, 0.0])
    d2 = np.array([0.3, -0.5, 0.8]); d2 /= np.linalg.norm(d2)
    e2 = np.cross(d2, [0, 0, 1.0]); e2 /= np.linalg.norm(e2)
    return [d1, d2], [e1, e2]


def _oracle_box_matvec(mat, eps, dx, k, d, e, x):
    S = physics.ldr_S(d, e)
    alphas = [physics.alpha_ldr(ep, k, dx, S) for ep in eps]
    ainv = operator.alpha_inv_box(mat, alphas)
    counts = np.bincount(mat.reshape(-1), minlength=len(eps) + 1)[1:]
    at = 1.0 / alphas[int(np.argmax(counts))] if counts.sum() else 1.0 / alphas[0]
    return operator.fft_matvec(x, mat, ainv, at, k, dx), at


@pytest.mark.gpu
@pytest.mark.parametrize("box", BOXES)
def test_matvec_parity(box):
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
    want = np.stack([_oracle_box_matvec(mat, eps, dx, k, dirs[r], pols[r], x[r])[0] for r in range(2)])
    y128 = plan.matvec(to_dev(x)).cpu().numpy()
    assert rel_err(y128, want) < 1e-10
    y64 = plan.matvec(to_dev(x, torch.complex64)).cpu().numpy()
    assert rel_err(y64, want) < 2e-5


@pytest.mark.gpu
def test_matvec_all_air_and_single_voxel():
    dda = dda_module()
    dx, k = 0.5, 1.0
    d, e = [0, 0, 1.0], [1.0, 0, 0]
    # all air: y = alpha_tilde^{-1} x
    mat = np.zeros((4, 4, 4), dtype=np.uint8)
    plan = dda.Plan(to_dev(mat, torch.uint8), [2.25], dx, k)
    plan.set_incidence([d], [e])
    x = random_field((1, 3, 4, 4, 4), np.random.default_rng(1))
    y = plan.matvec(to_dev(x)).cpu().numpy()
    at = 1.0 / physics.alpha_ldr(2.25, k, dx, 0.0)
    assert rel_err(y, at * x) < 1e-14
    # one voxel: no interaction, y = alpha^{-1} x
    mat1 = np.ones((1, 1, 1), dtype=np.uint8)
    plan1 = dda.Plan(to_dev(mat1, torch.uint8), [2.25], dx, k)
    plan1.set_incidence([d], [e])
    x1 = random_field((1, 3, 1, 1, 1), np.random.default_rng(2))
    y1 = plan1.matvec(to_dev(x1)).cpu().numpy()
    assert rel_err(y1, at * x1) < 1e-14


@pytest.mark.gpu
@pytest.mark.parametrize("box", BOXES)
def test_precond_apply_parity(box):
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
    want = []
    for r in range(2):
        p = Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[r], e=pols[r])
        want.append(p.precond3()(v[r]))
    want = np.stack(want)
    z128 = plan.precond_apply(to_dev(v)).cpu().numpy()
    assert rel_err(z128, want) < 1e-10
    z64 = plan.precond_apply(to_dev(v, torch.complex64)).cpu().numpy()
    assert rel_err(z64, want) < 2e-5


@pytest.mark.gpu
def test_incident_field_parity():
    dda = dda_module()
    l, m, n = 16, 8, 4
    dx, k = 0.2, 3.0
    mat = hex_prism_mask(l, m, n, dx, 1.5, 1.0)
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.7], dx, k, max_rhs=2)
    plan.set_incidence(dirs, pols)
    b = plan.incident_field().cpu().numpy()
    for r in range(2):
        p = Problem(mat=mat, dx=dx, k=k, eps=[1.7], d=dirs[r], e=pols[r])
        assert rel_err(b[r], p.rhs()) < 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("box", [(4, 4, 4), (8, 4, 2), (16, 8, 1), (2, 32, 16), (16, 16, 16)])
def test_precond_apply_parity_strang(box):
    """3-level preconditioner with Strang's circulant on every level."""
    dda = dda_module()
    l, m, n = box
    rng = np.random.default_rng(500 + sum(box))
    mat = hex_prism_mask(l, m, n, 2.0 / max(l, m), 1.0, 2.0)
    if mat.sum() == 0:
        mat[0, 0, 0] = 1
    dx, k = 2.0 / max(l, m), 2.2
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2, circulant="strang")
    plan.set_incidence(dirs, pols)
    plan.precond_build()
    v = random_field((2, 3, n, m, l), rng)
    want = np.stack([Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[r], e=pols[r])
                     .precond3(kind="strang")(v[r]) for r in range(2)])
    assert rel_err(plan.precond_apply(to_dev(v)).cpu().numpy(), want) < 1e-10
    assert rel_err(plan.precond_apply(to_dev(v, torch.complex64)).cpu().numpy(), want) < 2e-5


@pytest.mark.gpu
@pytest.mark.late(1)
def test_operator_parity_z256():
    """The preconditioner's z pass at transform length 256 and the matvec's at
    512 (the 256^3 solve's lengths), on a thin 4 x 4 x 256 box, vs the oracle."""
    dda = dda_module()
    l, m, n = 4, 4, 256
    rng = np.random.default_rng(256)
    mat = np.ones((n, m, l), dtype=np.uint8)
    mat[rng.random((n, m, l)) < 0.3] = 0
    dx, k = 0.05, 2.0
    dirs, pols = _incidences()
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2)
    plan.set_incidence(dirs, pols)
    plan.precond_build()
    v = random_field((2, 3, n, m, l), rng)
    want = np.stack([Problem(mat=mat, dx=dx, k=k, eps=[1.31 ** 2], d=dirs[r], e=pols[r])
                     .precond3()(v[r]) for r in range(2)])
    assert rel_err(plan.precond_apply(to_dev(v)).cpu().numpy(), want) < 1e-10
    assert rel_err(plan.precond_apply(to_dev(v, torch.complex64)).cpu().numpy(), want) < 2e-5
    wantm = np.stack([_oracle_box_matvec(mat, [1.31 ** 2], dx, k, dirs[r], pols[r], v[r])[0]
                      for r in range(2)])
    assert rel_err(plan.matvec(to_dev(v)).cpu().numpy(), wantm) < 1e-10
    assert rel_err(plan.matvec(to_dev(v, torch.complex64)).cpu().numpy(), wantm) < 2e-5
