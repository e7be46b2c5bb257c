"""Host logic of bench.py's roofline line, on the CPU: the committed ncu
summary is used only while the CUDA sources still hash to the value it
records, and the reported traffic is the launch-weighted mean of its
per-box figures over the profiled step."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_summary_guarded_by_source_hash(monkeypatch):
    cur = bench.traffic_from_profiles("mv_z_mul")
    if cur is not None:
        assert set(cur) >= {"64x64x32", "64x64x64", "64x64x128"}
        assert all(v > 0 for v in cur.values())
    monkeypatch.setattr(bench, "source_hash", lambda: "0" * 16)
    assert bench.traffic_from_profiles("mv_z_mul") is None
    assert bench.traffic_from_profiles("no_such_kernel") is None


class _FakeRunner:
    """Two boxes; the dominant class 'a' has 3 and 1 launches on them."""

    def __init__(self):
        self.profile, self.prof = False, []

    def step(self):
        assert self.profile
        self.prof.append((SimpleNamespace(dims=(4, 4, 2)),
                          {"a": (3.0, 3, 3e9), "b": (1.0, 2, 1e9)}))
        self.prof.append((SimpleNamespace(dims=(4, 4, 4)),
                          {"a": (2.0, 1, 2e9), "b": (0.5, 1, 5e8)}))


def test_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "traffic_from_profiles",
                        lambda k: {"4x4x2": 100.0, "4x4x4": 300.0} if k == "a" else None)
    r = bench.roofline(_FakeRunner(), 1000.0, "measured")
    assert r["kernel"] == "a"
    # 5e9 algorithmic bytes in 5 ms over 4 launches
    assert r["achieved"] == pytest.approx(1000.0)
    assert r["frac"] == pytest.approx(1.0)
    assert r["avg_launch_us"] == pytest.approx(1250.0)
    assert r["algorithmic_bytes_per_launch"] == round(5e9 / 4)
    assert r["traffic"] == round((3 * 100.0 + 1 * 300.0) / 4)
    assert r["share_of_profiled_kernel_time"]["a"] == pytest.approx(5.0 / 6.5, abs=1e-4)


def test_roofline_traffic_null_without_summary(monkeypatch):
    monkeypatch.setattr(bench, "traffic_from_profiles", lambda k: None)
    assert bench.roofline(_FakeRunner(), 1000.0, "measured")["traffic"] is None


def test_cufft_comparison_runs_on_cpu():
    # the cuFFT side of the matvec comparison, on the CPU backend of torch.fft:
    # same code, tiny box, just that it runs and times something
    ms = bench.cufft_convolution_ms(4, 4, 2, 2, "cpu", reps=2, warmup=1)
    assert ms > 0
