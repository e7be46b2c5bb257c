"""Launch schedules and the autotuner: every schedule (register-resident or
all-shared-memory z pass, with or without programmatic dependent launch, the
z pass's registers bounded to three blocks per SM or not) gives the oracle's
operator on the 64 x 64 x {32, 64} boxes of the bench's prism sweep (z
transforms of length 64 and 128, where the z kernels differ); dda_autotune
times all eight, keeps the fastest and serves the next plan of the same shape
from its table."""
import ctypes

import numpy as np
import pytest
import torch

from dda_inputs import random_field
from gpu_util import dda_module, rel_err, to_dev
from oracle import operator, physics


def _oracle_matvec(mat, eps, dx, k, d, e, x):
    S = physics.ldr_S(d, e)
    alphas = [physics.alpha_ldr(ep, k, dx, S) for ep in eps]
    ainv = operator.alpha_inv_box(mat, alphas)
    counts = np.bincount(mat.reshape(-1), minlength=len(eps) + 1)[1:]
    at = 1.0 / alphas[int(np.argmax(counts))]
    return operator.fft_matvec(x, mat, ainv, at, k, dx)


@pytest.mark.gpu
@pytest.mark.late(4)
@pytest.mark.parametrize("n", [32, 64])
def test_every_schedule_gives_the_operator_and_autotune(n):
    dda = dda_module()
    l = m = 64
    rng = np.random.default_rng(100 + n)
    mat = (rng.random((n, m, l)) < 0.6).astype(np.uint8)
    mat[rng.random((n, m, l)) < 0.2] *= 2
    eps = [1.31 ** 2, (1.6 + 0.05j) ** 2]
    dx, k = 0.3, 1.7
    d = np.array([0.3, -0.5, 0.8]); d /= np.linalg.norm(d)
    e = np.cross(d, [0, 0, 1.0]); e /= np.linalg.norm(e)
    x = random_field((1, 3, n, m, l), rng)
    want = _oracle_matvec(mat, eps, dx, k, d, e, x[0])[None]

    mat_d = to_dev(mat, torch.uint8)
    plan = dda.Plan(mat_d, eps, dx, k, max_rhs=1)
    plan.set_incidence([d], [e])
    assert plan.schedule() == {"rr_z": True, "pdl": False, "graph": True, "z_occ": True}
    x64, x128 = to_dev(x, torch.complex64), to_dev(x)
    for rr_z in (True, False):
        for pdl in (True, False):
            for z_occ in (True, False):
                plan.set_schedule(rr_z, pdl, z_occ=z_occ)
                assert plan.schedule() == {"rr_z": rr_z, "pdl": pdl, "graph": True, "z_occ": z_occ}
                assert rel_err(plan.matvec(x64).cpu().numpy(), want) < 2e-5
                assert rel_err(plan.matvec(x128).cpu().numpy(), want) < 1e-10
    bad = dda.Schedule(2, 1, 1, 1)
    assert dda.STATUS[dda._lib.dda_schedule_set(plan.handle, ctypes.byref(bad))] == \
        "DDA_ERR_INVALID_ARG"

    rep = plan.autotune(reps=3, force=True)
    assert not rep["cached"] and len(rep["timed"]) == 8
    assert all(ms > 0 for _, ms in rep["timed"])
    assert len({(s["rr_z"], s["pdl"], s["z_occ"]) for s, _ in rep["timed"]}) == 8
    assert rep["chosen"] == min(rep["timed"], key=lambda t: t[1])[0]
    assert plan.schedule() == rep["chosen"]
    assert rel_err(plan.matvec(x64).cpu().numpy(), want) < 2e-5

    plan2 = dda.Plan(mat_d, eps, dx, k, max_rhs=1)
    plan2.set_incidence([d], [e])
    rep2 = plan2.autotune(reps=3)
    assert rep2["cached"] and rep2["timed"] == [] and rep2["chosen"] == rep["chosen"]
    assert plan2.schedule() == rep["chosen"]
    with pytest.raises(dda.DDAError):
        plan2.autotune(reps=0)
