"""The C ABI library: symbols, workspace sizing and argument checks (no GPU needed)."""
import ctypes
from types import SimpleNamespace
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dda():
    from paper_1903_09802_gb300.build import build
    build()
    from paper_1903_09802_gb300 import dda as mod
    return mod


def _declared():
    text = open(os.path.join(ROOT, "include", "dda.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dda_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dda_plan_create", "dda_matvec", "dda_precond_build", "dda_solve",
              "dda_cross_sections", "dda_workspace_size", "dda_precond_apply"):
        assert n in names


def test_library_exports_every_declared_symbol(dda):
    lib = dda.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) == set(dda.EXPORTS)


def test_workspace_size_checks(dda):
    ok = dda.workspace_size(16, 16, 16, 0.125, 5.0, 1, 2, 50)
    assert ok > 0
    assert dda.workspace_size(32, 16, 16, 0.125, 5.0, 1, 2, 50) > ok
    assert dda.workspace_size(16, 16, 16, 0.125, 5.0, 1, 2, 0) < ok
    only64 = dda.workspace_size(16, 16, 16, 0.125, 5.0, 1, 2, 50, dda.PLAN_C64)
    assert 0 < only64 < ok
    for bad in [(15, 16, 16), (22, 16, 16), (16, 0, 16), (1024, 2, 2)]:
        assert dda.workspace_size(*bad, 0.125, 5.0) == 0
        err = dda.last_error()
        assert "power" in err or ">=" in err or "at most 512" in err, err
    # mixed-radix boxes (even 7-smooth edges) are taken
    assert dda.workspace_size(12, 16, 16, 0.125, 5.0) > 0
    assert dda.workspace_size(96, 96, 96, 0.125, 5.0) > 0
    assert dda.workspace_size(8, 8, 8, -1.0, 5.0) == 0
    assert dda.workspace_size(8, 8, 8, 0.1, 5.0, 0) == 0
    assert dda.workspace_size(8, 8, 8, 0.1, 5.0, 1, 1, 0, 0) == 0


def test_plan_create_argument_errors(dda):
    lib = dda.lib()
    desc = dda.PlanDesc(8, 8, 8, 0.25, 2.0, 1, 1, 10, 3)
    need = lib.dda_workspace_size(ctypes.byref(desc))
    eps = (ctypes.c_double * 2)(1.7161, 0.0)
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every check fails first
    st = lib.dda_plan_create(ctypes.byref(h), ctypes.byref(desc), fake, eps, fake, need - 1, None)
    assert dda.STATUS[st] == "DDA_ERR_WORKSPACE"
    st = lib.dda_plan_create(ctypes.byref(h), ctypes.byref(desc), fake, eps, ctypes.c_void_p((1 << 20) + 8), need, None)
    assert dda.STATUS[st] == "DDA_ERR_WORKSPACE"  # misaligned
    st = lib.dda_plan_create(ctypes.byref(h), ctypes.byref(desc), None, eps, fake, need, None)
    assert dda.STATUS[st] == "DDA_ERR_INVALID_ARG"
    # edges: odd, a prime factor above 7, above 512 (powers of two and even
    # 7-smooth numbers are taken)
    for edge in (9, 22, 210, 1024):
        bad = dda.PlanDesc(8, edge, 8, 0.25, 2.0, 1, 1, 10, 3)
        st = lib.dda_plan_create(ctypes.byref(h), ctypes.byref(bad), fake, eps, fake, need, None)
        assert dda.STATUS[st] == "DDA_ERR_UNSUPPORTED_SIZE", edge
        assert not h.value
    for edge in (6, 96, 200, 252):
        ok = dda.PlanDesc(8, edge, 8, 0.25, 2.0, 1, 1, 10, 3)
        assert lib.dda_workspace_size(ctypes.byref(ok)) > 0, edge


def test_null_plan_is_rejected(dda):
    lib = dda.lib()
    assert dda.STATUS[lib.dda_matvec(None, 0, 1, None, None, None)] == "DDA_ERR_INVALID_ARG"
    assert dda.STATUS[lib.dda_precond_build(None, None)] == "DDA_ERR_INVALID_ARG"
    assert dda.STATUS[lib.dda_solve(None, 1, None, None, None, None, None)] == "DDA_ERR_INVALID_ARG"
    sched = dda.Schedule(1, 1)
    assert dda.STATUS[lib.dda_schedule_set(None, ctypes.byref(sched))] == "DDA_ERR_INVALID_ARG"
    assert dda.STATUS[lib.dda_schedule_get(None, ctypes.byref(sched))] == "DDA_ERR_INVALID_ARG"
    assert dda.STATUS[lib.dda_autotune(None, 1, 1, None, None, 5, 0, None, None)] == \
        "DDA_ERR_INVALID_ARG"
    lib.dda_plan_destroy(None)


def test_workspace_options_validated():
    from paper_1903_09802_gb300 import dda
    base = dda.workspace_size(16, 16, 8, 0.125, 5.0, 1, 2, 50)
    assert dda.workspace_size(16, 16, 8, 0.125, 5.0, 1, 2, 50, precond2=1) > base
    assert dda.workspace_size(16, 16, 8, 0.125, 5.0, 1, 2, 50, circulant="strang") == base
    desc = dda.PlanDesc(16, 16, 8, 0.125, 5.0, 1, 2, 50, 3, 0, 2)  # circulant 2: unknown
    assert dda._lib.dda_workspace_size(ctypes.byref(desc)) == 0
    desc = dda.PlanDesc(16, 16, 8, 0.125, 5.0, 1, 2, 50, 3, 4, 0)  # precond2 4: unknown
    assert dda._lib.dda_workspace_size(ctypes.byref(desc)) == 0
    # Toeplitz level x on a 16 x 16 x 8 box: (8/2+1)(16/2+1) blocks of 48^2
    # instead of (16/2+1)^2 blocks of 24^2, plus the relabelled mask
    zsize = dda.workspace_size(16, 16, 8, 0.125, 5.0, 1, 2, 50, precond2="z")
    xsize = dda.workspace_size(16, 16, 8, 0.125, 5.0, 1, 2, 50, precond2="x")
    assert xsize - zsize >= (5 * 9 * 48 ** 2 - 81 * 24 ** 2) * 8


def test_toeplitz_axis_choice():
    from paper_1903_09802_gb300 import dda
    assert dda.toeplitz_axis_for(64, 64, 64) == "z"      # cube: the paper's level
    assert dda.toeplitz_axis_for(64, 64, 4) == "z"       # plate
    assert dda.toeplitz_axis_for(64, 64, 128) == "x"     # long prism along z
    assert dda.toeplitz_axis_for(64, 32, 128) == "y"
    assert dda.toeplitz_axis_for(16, 64, 64) == "x"
    z = dda.workspace_size(64, 64, 128, 0.1, 5.0, 1, 1, 0, precond2="z")
    auto = dda.workspace_size(64, 64, 128, 0.1, 5.0, 1, 1, 0, precond2="auto")
    x = dda.workspace_size(64, 64, 128, 0.1, 5.0, 1, 1, 0, precond2="x")
    assert auto == x < z


def test_autotune_report_marshalling(monkeypatch):
    # Plan.autotune's marshalling of dda_tune_report_t, with the C call replaced
    # by one that fills the report as the library does (no GPU needed)
    import torch
    from paper_1903_09802_gb300 import dda

    def fake_autotune(h, prec, nrhs, x, y, reps, flags, rep_ref, stream):
        rep = rep_ref._obj
        rep.ncand = 4
        for c in range(4):
            rep.cand[c].rr_z, rep.cand[c].pdl = int(c & 1 == 0), int(c & 2 == 0)
            rep.cand[c].graph, rep.cand[c].z_occ = 1, 1
            rep.ms_per_matvec[c] = [0.3, 0.2, 0.4, 0.5][c]
        rep.chosen = rep.cand[1]
        rep.cached = 0
        assert prec == dda.C64 and nrhs == 2 and reps == 7 and flags == 1
        return 0

    monkeypatch.setattr(dda, "_lib", SimpleNamespace(dda_autotune=fake_autotune))
    monkeypatch.setattr(dda, "_stream", lambda: None)
    plan = dda.Plan.__new__(dda.Plan)
    plan._h = None
    plan.nrhs = 2
    plan.incident_field = lambda n: torch.ones((n, 3, 2, 2, 2), dtype=torch.complex128)
    rep = plan.autotune(reps=7, force=True)
    assert rep["chosen"] == {"rr_z": False, "pdl": True, "graph": True, "z_occ": True} \
        and not rep["cached"]
    assert [t[1] for t in rep["timed"]] == pytest.approx([0.3, 0.2, 0.4, 0.5])
    assert rep["timed"][3][0] == {"rr_z": False, "pdl": False, "graph": True, "z_occ": True}
    plan._h = None  # nothing to destroy


def _fake_plan(dda, shape=(8, 4, 2)):
    """A Plan object with no library handle: enough for the binding's own
    argument checks, which must raise before any pointer reaches the library."""
    import torch
    p = object.__new__(dda.Plan)
    l, m, n = shape
    p.mat = torch.zeros((n, m, l), dtype=torch.uint8)
    p.shape = shape
    p._h = None
    p.nrhs = 2
    return p


def test_binding_rejects_bad_out_before_any_launch(dda, monkeypatch):
    import torch

    def boom(*a, **k):  # any call into the library would be a launch
        raise AssertionError("library called")

    for name in ("dda_matvec", "dda_precond_apply", "dda_precond2_apply",
                 "dda_precond_apply_noalloc", "dda_fft3d", "dda_cross_sections",
                 "dda_ext_gradient", "dda_solve"):
        monkeypatch.setattr(dda._lib, name, boom)
    p = _fake_plan(dda)
    v = torch.zeros(p.field_shape(2), dtype=torch.complex64)
    bad_outs = [torch.zeros(p.field_shape(1), dtype=torch.complex64),         # too small
                torch.zeros(p.field_shape(2), dtype=torch.complex128),        # other dtype
                torch.zeros((2, 3, 2, 4, 16), dtype=torch.complex64)[..., ::2],  # strided
                "not a tensor"]
    for apply in (p.matvec, p.precond_apply, p.precond2_apply, p.precond_apply_noalloc):
        for out in bad_outs:
            with pytest.raises((TypeError, ValueError)):
                apply(v, out)
    with pytest.raises(ValueError):
        p.precond_apply_noalloc(v, None)
    with pytest.raises(ValueError):
        p.matvec(v, v)                                       # y must not alias x
    with pytest.raises(ValueError):
        p.precond_apply(torch.zeros((2, 3, 2, 4, 4), dtype=torch.complex64))  # wrong box
    with pytest.raises(TypeError):
        p.precond_apply(torch.zeros(p.field_shape(2), dtype=torch.float32))
    with pytest.raises(TypeError):
        p.cross_sections(v)                                  # solutions are complex128
    with pytest.raises(ValueError):
        p.fft3d(torch.zeros((1, 2, 4, 4), dtype=torch.complex64))
    with pytest.raises(ValueError):
        p.ext_gradient_from(torch.zeros(p.field_shape(2), dtype=torch.complex128),
                            torch.zeros(p.field_shape(1), dtype=torch.complex128))
    with pytest.raises(ValueError):
        p.solve(b=torch.zeros(p.field_shape(1)[:-1] + (3,), dtype=torch.complex128))
