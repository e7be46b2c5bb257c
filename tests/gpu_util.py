"""Helpers shared by the GPU parity tests (oracle inputs -> CUDA library)."""
import numpy as np
import pytest
import torch


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dda_module():
    need_gpu()
    from paper_1903_09802_gb300.build import build
    build()
    from paper_1903_09802_gb300 import dda
    return dda


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def rel_err(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))
