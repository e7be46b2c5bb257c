"""The per-thread launch schedule (dda_schedule_set / dda_autotune choose
it per plan; each entry point installs its plan's schedule with a scope),
checked on the host: scopes nest and restore, other threads keep theirs, and
the switches the launch code reads follow the scope.  The GPU test of every
schedule's results is tests/test_gpu_autotune.py."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_schedule_scopes(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "schedule_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(HERE, "native", "schedule_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    env = {k: v for k, v in os.environ.items() if k not in ("DDA_PDL", "DDA_RR_FFT3C")}
    out = subprocess.run([exe], check=True, capture_output=True, text=True, env=env).stdout
    seen = {name: (int(a), int(b)) for name, a, b in (ln.split() for ln in out.splitlines())}
    assert seen == {"default": (1, 0), "outer": (0, 1), "inner": (1, 0),
                    "other_thread": (1, 0), "outer_again": (0, 1), "restored": (1, 0)}
    # the environment switches force the plain forms whatever the schedule
    env["DDA_PDL"] = "0"
    out = subprocess.run([exe], check=True, capture_output=True, text=True, env=env).stdout
    assert all(ln.split()[2] == "0" for ln in out.splitlines())
