"""dda_precond_apply_noalloc, the preconditioner apply that allocates nothing.

Callers that cannot allocate device memory while they run (a host with
device memory fixed at start-up, a framework owning every byte of the device
through its own pool) use this entry point; its scratch is a fixed array
inside the library.  This file is collected last so
that a failure here comes after every other test has run.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from dda_inputs import hex_prism_mask, random_field
from gpu_util import dda_module, rel_err, to_dev

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _plan(dda):
    l, m, n = 16, 32, 8
    dx, k = 2.0 / 32, 4.0
    mat = hex_prism_mask(l, m, n, dx, 0.5, 0.5)
    plan = dda.Plan(to_dev(mat, torch.uint8), [1.31 ** 2], dx, k, max_rhs=2)
    plan.set_incidence([[0, 0, 1.0], [0.6, 0, 0.8]], [[1.0, 0, 0], [0, 1.0, 0]])
    plan.precond_build()
    return plan, (l, m, n)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_noalloc_apply_matches_workspace_apply(prec):
    dda = dda_module()
    plan, (l, m, n) = _plan(dda)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    tol = 1e-10 if prec == "c128" else 2e-5
    rng = np.random.default_rng(11)
    for call in range(2):  # two calls in a row: the shared scratch is reused
        v = to_dev(random_field((2, 3, n, m, l), rng), dt)
        want = plan.precond_apply(v).cpu().numpy()
        out = torch.empty_like(v)
        plan.precond_apply_noalloc(v, out)
        got = out.cpu().numpy()
        assert rel_err(got, want) < tol, (prec, call)


# Run in a child process with a context of its own: the device's free memory
# is process-wide, and in the test process other tests' objects (plans and
# their CUDA graphs, collected by Python's garbage collector at any moment)
# move it independently of the call being measured.
_CHILD = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import gc
import numpy as np, torch
from gpu_util import dda_module, to_dev
from dda_inputs import random_field
from test_zz_no_alloc import _plan
dda = dda_module()
plan, (l, m, n) = _plan(dda)
rng = np.random.default_rng(5)
for dt in (torch.complex128, torch.complex64):
    v = to_dev(random_field((2, 3, n, m, l), rng), dt)
    plan.precond_apply(v)
    out = torch.empty_like(v)
    for call in range(2):
        gc.collect()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        plan.precond_apply_noalloc(v, out)
        torch.cuda.synchronize()
        print(dt, call, free0 - torch.cuda.mem_get_info()[0])
"""


@pytest.mark.gpu
def test_noalloc_apply_allocates_nothing():
    """The call's whole contract: the device's free memory does not move,
    on the first call (plan creation loaded the array) as on the second."""
    dda_module()  # builds the library if needed
    code = _CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln.split() for ln in r.stdout.splitlines() if ln.startswith("torch.")]
    assert len(lines) == 4, r.stdout
    for dt, call, delta in lines:
        assert int(delta) == 0, (dt, call, delta)


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
