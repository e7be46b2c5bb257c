"""The double-float arithmetic of the complex128 matvec (dfloat.cuh), checked
on the host: conversion from double keeps 48 bits, and +, -, * of
double-float values are accurate to a few units of 2^-48 relative (the sums
in double of the exact operand values are exact or within 2^-53 here).  The
FFT kernels built on these operations are checked on the GPU against the
FP64 oracle at 1e-10."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_double_float_operations(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dfloat_check")
    # the header's kernels are compiled for the library's target; only host code runs
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "native", "dfloat_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    e_rt, e_add, e_sub, e_mul = map(float, out)
    assert e_rt <= 2.0 ** -48
    assert e_add <= 4 * 2.0 ** -48 and e_sub <= 4 * 2.0 ** -48
    assert e_mul <= 4 * 2.0 ** -48
