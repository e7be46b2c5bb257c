"""dda_precond_apply_noalloc, the preconditioner apply that allocates nothing.

Callers that cannot allocate device memory while they run (a host with
device memory fixed at start-up, a framework owning every byte of the device
through its own pool) use this entry point; its scratch is a fixed array
inside the library.  This file is collected last so
that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask, random_field
from gpu_util import dda_module, rel_err, to_dev


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_apply_matches_workspace_apply(prec):
    dda = dda_module()
    l, m, n = 16, 32, 8
    dx, k = 2.0 / 32, 4.0
    mat = hex_prism_mask(l, m, n, dx, 0.5, 0.5)
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2)
    plan.set_incidence([[0, 0, 1.0], [0.6, 0, 0.8]], [[1.0, 0, 0], [0, 1.0, 0]])
    plan.precond_build()
    dt = torch.complex128 if prec == "c128" else torch.complex64
    tol = 1e-10 if prec == "c128" else 2e-5
    rng = np.random.default_rng(11)
    for call in range(2):  # two calls in a row: the shared scratch is reused
        v = to_dev(random_field((2, 3, n, m, l), rng), dt)
        want = plan.precond_apply(v).cpu().numpy()
        out = torch.empty_like(v)
        # the call's whole contract: the device's free memory does not move,
        # on the first call as on the second (plan creation loaded the array)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        plan.precond_apply_noalloc(v, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before, (prec, call)
        got = out.cpu().numpy()
        assert rel_err(got, want) < tol, (prec, call)


@pytest.mark.gpu
def test_noalloc_apply_rejects_oversize():
    dda = dda_module()
    l = m = n = 128
    mat = torch.zeros((n, m, l), dtype=torch.uint8, device="cuda")
    plan = dda.Plan(mat, [1.7], 0.1, 1.0, max_rhs=1)
    plan.set_incidence([[0, 0, 1.0]], [[1.0, 0, 0]])
    plan.precond_build()
    v = torch.zeros((1, 3, n, m, l), dtype=torch.complex128, device="cuda")
    with pytest.raises(dda.DDAError) as e:
        plan.precond_apply_noalloc(v, torch.empty_like(v))
    assert "DDA_ERR_WORKSPACE" in str(e.value) and "static scratch" in str(e.value)


@pytest.mark.gpu
def test_noalloc_apply_rejects_mixed_radix_box():
    """Mixed-radix boxes (even 7-smooth edges) are refused before any launch:
    their kernels carry a local stack frame whose first launch may make the
    driver enlarge the context's local-memory reservation."""
    dda = dda_module()
    l, m, n = 12, 8, 8
    mat = torch.ones((n, m, l), dtype=torch.uint8, device="cuda")
    plan = dda.Plan(mat, [1.7], 0.1, 1.0, max_rhs=1)
    plan.set_incidence([[0, 0, 1.0]], [[1.0, 0, 0]])
    plan.precond_build()
    v = torch.zeros((1, 3, n, m, l), dtype=torch.complex128, device="cuda")
    with pytest.raises(dda.DDAError) as e:
        plan.precond_apply_noalloc(v, torch.empty_like(v))
    assert "DDA_ERR_UNSUPPORTED_SIZE" in str(e.value)
