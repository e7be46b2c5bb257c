"""K3: the shared-memory Stockham FFT against numpy.fft (3-D, both precisions)."""
import numpy as np
import pytest
import torch

from dda_inputs import random_field
from gpu_util import dda_module, rel_err, to_dev

SHAPES = [(1, 1, 1), (2, 4, 8), (16, 16, 16), (32, 8, 4), (64, 2, 128), (512, 2, 4), (8, 512, 2),
          (4, 2, 512), (128, 64, 32)]


@pytest.mark.gpu
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_fft3d_matches_numpy(shape, prec):
    dda = dda_module()
    l, m, n = shape
    mat = torch.ones((n, m, l), dtype=torch.uint8, device="cuda")
    plan = dda.Plan(mat, [2.0], 0.1, 1.0, precisions=dda.PLAN_C128 | dda.PLAN_C64)
    rng = np.random.default_rng(l * 7 + m * 3 + n)
    a = random_field((3, n, m, l), rng)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    tol = 1e-12 if prec == "c128" else 3e-6
    t = to_dev(a, dt)
    plan.fft3d(t)
    want = np.fft.fftn(a, axes=(1, 2, 3))
    assert rel_err(t.cpu().numpy(), want) < tol
    plan.fft3d(t, inverse=True)
    assert rel_err(t.cpu().numpy(), a) < tol
