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
    monkeypatch.setattr(bench, "source_hash", lambda files=None: "0" * 16)
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


class _FakeReplay:
    """Replays of the class 'mv_z_mul': 20 launches of 0.1 ms (1e8 bytes each)
    on box 4x4x2 and of 0.3 ms (3e8 bytes each) on 4x4x4."""

    def replay_matvec(self, dims, reps):
        per = {(4, 4, 2): (0.1, 1e8), (4, 4, 4): (0.3, 3e8)}[dims]
        return {"mv_z_mul": (per[0] * reps, reps, per[1] * reps)}


def test_matvec_replay_weights_boxes_by_step_launches():
    # the step launched the class 3 times on 4x4x2 and once on 4x4x4
    r = bench.matvec_replay(_FakeReplay(), "mv_z_mul", {(4, 4, 2): 3, (4, 4, 4): 1, (8, 8, 8): 0})
    assert r["avg_launch_us"] == pytest.approx(1e3 * (3 * 0.1 + 0.3) / 4)
    # (3 * 1e8 + 3e8) / 4 bytes per launch over 150 us
    assert r["achieved"] == pytest.approx(1.5e8 / 150e-6 / 1e9, rel=1e-3)
    assert r["us_per_launch_by_box"] == {"4x4x2": 100.0, "4x4x4": 300.0}


def test_roofline_traffic_null_without_summary(monkeypatch):
    monkeypatch.setattr(bench, "traffic_from_profiles", lambda k: None)
    assert bench.roofline(_FakeRunner(), 1000.0, "measured")["traffic"] is None


def test_cufft_comparison_runs_on_cpu():
    # the cuFFT side of the matvec comparison, on the CPU backend of torch.fft:
    # same code, tiny box, just that it runs and times something
    ms = bench.cufft_convolution_ms(4, 4, 2, 2, "cpu", reps=2, warmup=1)
    assert ms > 0


class _FakeRes:
    def __init__(self, nrhs):
        import numpy as np
        self.iters = [3] * nrhs
        self.cycles = [1] * nrhs
        self.converged = [True] * nrhs
        self.rel_resid = [1e-7] * nrhs
        self.history = [np.array([1.0, 1e-3, 1e-7])] * nrhs
        self.graph = True
        self.status = 0
        self.x = None


class _FakePlan:
    """Stands in for dda.Plan on the CPU: records calls, computes nothing."""

    def __init__(self, mat, eps, dx, k, max_rhs=1, krylov_m=0, precond2=False, **kw):
        self.shape = tuple(mat.shape)
        self.precond2 = precond2
        self.nrhs = 0

    def set_incidence(self, dirs, pols):
        self.nrhs = len(dirs)

    def precond_build(self):
        pass

    def precond2_build(self):
        assert self.precond2

    def solve(self, **kw):
        assert kw["precond"] in (0, 2, 3) and (kw["precond"] != 2 or self.precond2)
        return _FakeRes(self.nrhs)

    def profile(self, on=True):
        pass

    def profile_read(self):
        return {"mv_z_mul": (1.0, 2, 1e9), "mv_x_fwd": (0.5, 2, 4e8)}

    def cross_sections(self, x):
        import numpy as np
        return np.tile([2.0, 0.5, 1.5], (self.nrhs, 1))

    def incident_field(self, nrhs):
        import torch
        n, m, l = self.shape
        return torch.ones((nrhs, 3, n, m, l), dtype=torch.complex128)

    def matvec(self, x, out=None):
        return x


class _FakeEvent:
    def __init__(self, **kw):
        pass

    def record(self, *a):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 1.0


def test_side_comparisons_run_with_a_stand_in_library(monkeypatch):
    # the Python of the guarded comparisons (2-level sweep, 128^3 precision pair,
    # cuFFT matvec), run against a stand-in library on the CPU so that a slip in
    # it shows here rather than as an error entry of the GPU run's JSON line
    import numpy as np
    import torch
    from paper_1903_09802_gb300 import dda as real
    fake = SimpleNamespace(Plan=_FakePlan, C64=real.C64, C128=real.C128, STATUS=real.STATUS,
                           precond_for=real.precond_for, BICGSTAB=real.BICGSTAB,
                           workspace_size=lambda *a, **k: 123,
                           solve_many=lambda plans, **kw: [_FakeRes(1) for _ in plans])
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    monkeypatch.setattr(bench, "cufft_convolution_ms", lambda *a, **k: 2.0)
    cases = [SimpleNamespace(dims=(4, 4, 2), eps=[1.31 ** 2], dx=0.5, k=1.0, nrhs=2,
                             dirs=[np.array([0, 0, 1.0])] * 2,
                             pols=[np.array([1.0, 0, 0]), np.array([0, 1.0, 0])])]
    runner = SimpleNamespace(dda=fake, cases=cases, masks=[torch.zeros((2, 4, 4), dtype=torch.uint8)],
                             dev="cpu")
    pol = bench.compare_policy(runner)
    row = pol["4x4x2 m=1.31+0.00j"]
    assert row["policy"] == "2-level" and row["none"]["ms_per_solve_with_setup"] >= 0
    assert isinstance(row["policy_beats_none"], bool)

    def step(inner="c64", **kw):
        return [([3, 3], [1e-7, 1e-7], None)]
    runner.step = step
    ps = bench.compare_precision_sweep(runner)
    assert ps["c128"]["max_rel_resid"] == 1e-7 and ps["c128_over_mixed"] > 0
    m178 = bench.compare_m178(runner)
    assert len(m178) == 3 and all(v["gmres_none"]["min_rel_resid"] == [1e-7, 1e-7]
                                  for v in m178.values())
    monkeypatch.setattr(_FakePlan, "cross_sections",
                        lambda self, x: np.tile([6.029132679, 1.38, 4.646511536], (1, 1)))
    tw = bench.compare_twin(runner)
    assert tw["c_ext_rel_err_vs_oracle"] < 1e-8 and tw["c_sca_rel_err_vs_oracle"] < 1e-8
    r128 = bench.roofline_128(runner, 1000.0, "measured")
    assert r128["passes"]["mv_z_mul"]["us_per_launch"] == 500.0
    ub = bench.compare_uneven_batch(runner, cap=5)
    assert ub["converged"] == 32 and len(ub["prisms (N, box edge, m)"]) == 32
    fft = bench.compare_fft(runner, reps=2)
    assert fft["4x4x2"]["speedup"] == 4.0  # 2 ms against 1 ms over 2 calls
    p128 = bench.compare_precision_128(runner)
    assert p128["c_ext_rel_diff"] == 0.0 and p128["c128"]["converged"]
