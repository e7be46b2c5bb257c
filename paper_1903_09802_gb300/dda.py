"""ctypes binding of libdda.so (the C ABI declared in include/dda.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory and the current CUDA stream.  Box
fields are complex tensors of shape (nrhs, 3, n, m, l) on the plan's device.
If the library is missing this module raises at import time; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdda.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1903_09802_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)

C128, C64 = 0, 1
GMRES, BICGSTAB = 0, 1
PLAN_C128, PLAN_C64 = 1, 2

STATUS = {
    0: "DDA_OK", 1: "DDA_ERR_INVALID_ARG", 2: "DDA_ERR_UNSUPPORTED_SIZE", 3: "DDA_ERR_WORKSPACE",
    4: "DDA_ERR_CUDA", 5: "DDA_ERR_NOT_CONVERGED", 6: "DDA_ERR_BREAKDOWN",
    7: "DDA_ERR_SINGULAR_PRECOND", 8: "DDA_ERR_NAN", 9: "DDA_ERR_TIMEOUT", 10: "DDA_ERR_NO_PRECOND",
}

CIRCULANTS = {"chan": 0, "strang": 1}  # preconditioner circulant: eq. 13 or Strang's


def toeplitz_axis_for(l: int, m: int, n: int) -> str:
    """The 2-level preconditioner's Toeplitz (dense) level for a box: the
    shortest edge, so the two longest levels are circulant (Section 5: for
    plates z, for prisms longer than wide an x or y level).  Ties go to z, then
    x: cubes keep the paper's choice, and a 64 x 64 x 128 prism gets x, which
    halves the dense blocks and measured 26% faster than z."""
    shortest = min(l, m, n)
    if n == shortest:
        return "z"
    return "x" if l == shortest else "y"


def precond_for(l: int, m: int, n: int) -> int:
    """Preconditioner policy for a box: the paper's 2-level form (3 returned
    as 2) for plate-like boxes, whose shortest edge is at most half of each
    of the other two (the Toeplitz level then is that short edge, and the
    circulant levels are the long ones: Section 3's setting), the 3-level form
    otherwise.  On the 64^3 sweep the 3-level form needs twice the iterations
    of the unpreconditioned solve on the 64 x 64 x 32 prism, where the 2-level
    one needs 0.6 times as many; on the cube and the long prism the 3-level
    form is faster once the 2-level build is counted."""
    dims = sorted((l, m, n))
    return 2 if 2 * dims[0] <= dims[1] else 3


def _precond2_code(v, dims=None) -> int:
    """2-level storage request: False (none), True or "z" (Toeplitz level z, the
    paper's), "x" or "y" (that level Toeplitz instead), "auto" (the shortest
    edge, toeplitz_axis_for)."""
    if v == "auto":
        v = toeplitz_axis_for(*dims)
    if v is False or v is None or v == 0:
        return 0
    if v is True or v == "z" or v == 1:
        return 1
    return {"x": 2, "y": 3}[v]

EXPORTS = ("dda_workspace_size", "dda_plan_create", "dda_set_incidence", "dda_incident_field",
           "dda_set_voxel_eps",
           "dda_matvec", "dda_precond_build", "dda_precond_apply", "dda_precond_apply_noalloc",
           "dda_precond2_build", "dda_precond2_apply",
           "dda_fft3d", "dda_solve", "dda_solve_many", "dda_ritz_shifts",
           "dda_cross_sections", "dda_adjoint_rhs", "dda_ext_gradient", "dda_profile_enable", "dda_profile_read", "dda_plan_destroy",
           "dda_schedule_set", "dda_schedule_get", "dda_autotune",
           "dda_last_error", "dda_launch_count")

PROFILE_NAMES = ("mv_x_fwd", "mv_y_fwd", "mv_z_mul", "mv_y_inv", "mv_x_inv", "pc_x_fwd", "pc_y_fwd",
                 "pc_z_solve", "pc_y_inv", "pc_x_inv", "gs_dots", "gs_update", "p2_block",
                 "mv128_x_fwd", "mv128_y_fwd", "mv128_z_mul", "mv128_y_inv", "mv128_x_inv",
                 "pc128_x_fwd", "pc128_y_fwd", "pc128_z_solve", "pc128_y_inv", "pc128_x_inv")


class DDAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class PlanDesc(ctypes.Structure):
    _fields_ = [("l", ctypes.c_int32), ("m", ctypes.c_int32), ("n", ctypes.c_int32),
                ("dx", ctypes.c_double), ("k", ctypes.c_double),
                ("n_materials", ctypes.c_int32), ("max_rhs", ctypes.c_int32),
                ("krylov_m", ctypes.c_int32), ("precisions", ctypes.c_int32),
                ("precond2", ctypes.c_int32), ("circulant", ctypes.c_int32),
                ("voxel_eps", ctypes.c_int32), ("rhs_chunk", ctypes.c_int32),
                ("krylov_c64", ctypes.c_int32), ("sstep", ctypes.c_int32)]


class Incidence(ctypes.Structure):
    _fields_ = [("dir", ctypes.c_double * 3), ("pol", ctypes.c_double * 3)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("inner_prec", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("reorth_eta", ctypes.c_double), ("method", ctypes.c_int32),
                ("history_cap", ctypes.c_int32), ("timeout_ns", ctypes.c_int64),
                ("h_history", ctypes.POINTER(ctypes.c_double))]


class RhsStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_resid", ctypes.c_double), ("reorth", ctypes.c_int32),
                ("history_len", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("ms", ctypes.c_float)]


class Schedule(ctypes.Structure):
    _fields_ = [("rr_z", ctypes.c_int32), ("pdl", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("z_occ", ctypes.c_int32)]


class TuneReport(ctypes.Structure):
    _fields_ = [("chosen", Schedule), ("cached", ctypes.c_int32), ("ncand", ctypes.c_int32),
                ("cand", Schedule * 8), ("ms_per_matvec", ctypes.c_float * 8)]


_vp = ctypes.c_void_p
_lib.dda_workspace_size.restype = ctypes.c_size_t
_lib.dda_workspace_size.argtypes = [ctypes.POINTER(PlanDesc)]
_lib.dda_plan_create.restype = ctypes.c_int
_lib.dda_plan_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(PlanDesc), _vp,
                                 ctypes.POINTER(ctypes.c_double), _vp, ctypes.c_size_t, _vp]
_lib.dda_set_incidence.restype = ctypes.c_int
_lib.dda_set_incidence.argtypes = [_vp, ctypes.c_int32, ctypes.POINTER(Incidence), _vp]
_lib.dda_set_voxel_eps.restype = ctypes.c_int
_lib.dda_set_voxel_eps.argtypes = [_vp, _vp, _vp]
_lib.dda_incident_field.restype = ctypes.c_int
_lib.dda_incident_field.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
_lib.dda_matvec.restype = ctypes.c_int
_lib.dda_matvec.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]
_lib.dda_precond_build.restype = ctypes.c_int
_lib.dda_precond_build.argtypes = [_vp, _vp]
_lib.dda_precond_apply.restype = ctypes.c_int
_lib.dda_precond_apply.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]
_lib.dda_solve_many.restype = ctypes.c_int
_lib.dda_solve_many.argtypes = [ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.dda_precond2_build.restype = ctypes.c_int
_lib.dda_precond2_build.argtypes = [_vp, _vp]
_lib.dda_precond2_apply.restype = ctypes.c_int
_lib.dda_precond2_apply.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]
_lib.dda_precond_apply_noalloc.restype = ctypes.c_int
_lib.dda_precond_apply_noalloc.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]
_lib.dda_fft3d.restype = ctypes.c_int
_lib.dda_fft3d.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32, _vp]
_lib.dda_solve.restype = ctypes.c_int
_lib.dda_solve.argtypes = [_vp, ctypes.c_int32, _vp, _vp, ctypes.POINTER(SolveOpts),
                           ctypes.POINTER(RhsStats), _vp]
_lib.dda_cross_sections.restype = ctypes.c_int
_lib.dda_cross_sections.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.POINTER(ctypes.c_double), _vp]
_lib.dda_adjoint_rhs.restype = ctypes.c_int
_lib.dda_adjoint_rhs.argtypes = [_vp, ctypes.c_int32, _vp, _vp]
_lib.dda_ext_gradient.restype = ctypes.c_int
_lib.dda_ext_gradient.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp]
_lib.dda_profile_enable.restype = ctypes.c_int
_lib.dda_profile_enable.argtypes = [_vp, ctypes.c_int32]
_lib.dda_profile_read.restype = ctypes.c_int
_lib.dda_profile_read.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int32]
_lib.dda_schedule_set.restype = ctypes.c_int
_lib.dda_schedule_set.argtypes = [_vp, ctypes.POINTER(Schedule)]
_lib.dda_schedule_get.restype = ctypes.c_int
_lib.dda_schedule_get.argtypes = [_vp, ctypes.POINTER(Schedule)]
_lib.dda_autotune.restype = ctypes.c_int
_lib.dda_autotune.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, ctypes.c_int32,
                              ctypes.c_int32, ctypes.POINTER(TuneReport), _vp]
_lib.dda_plan_destroy.restype = None
_lib.dda_plan_destroy.argtypes = [_vp]
_lib.dda_last_error.restype = ctypes.c_char_p
_lib.dda_last_error.argtypes = []
_lib.dda_ritz_shifts.restype = ctypes.c_int
_lib.dda_ritz_shifts.argtypes = [_vp, ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
_lib.dda_launch_count.restype = ctypes.c_int64
_lib.dda_launch_count.argtypes = []


def ritz_shifts(hraw: torch.Tensor, jlen: torch.Tensor, s: int) -> torch.Tensor:
    """dda_ritz_shifts: hraw (nrhs, m, m+1) complex128 CUDA tensor whose row j
    is Hessenberg column j; jlen (nrhs,) int32 CUDA.  Returns (nrhs, 8)
    complex128 shifts (the first s used)."""
    if (hraw.dtype != torch.complex128 or not hraw.is_cuda or hraw.dim() != 3 or
            hraw.shape[2] != hraw.shape[1] + 1 or not hraw.is_contiguous()):
        raise ValueError("hraw must be a contiguous (nrhs, m, m+1) complex128 CUDA tensor")
    if jlen.dtype != torch.int32 or jlen.shape != (hraw.shape[0],) or not jlen.is_cuda:
        raise ValueError("jlen must be an (nrhs,) int32 CUDA tensor")
    out = torch.zeros((hraw.shape[0], 8), dtype=torch.complex128, device=hraw.device)
    _check(_lib.dda_ritz_shifts(_ptr(hraw), hraw.shape[1], _ptr(jlen.contiguous()),
                                hraw.shape[0], int(s), _ptr(out), _stream()))
    return out


def launch_count() -> int:
    """Kernels launched by libdda.so in this process."""
    return int(_lib.dda_launch_count())


def lib():
    return _lib


def last_error() -> str:
    return _lib.dda_last_error().decode()


def _check(status: int):
    if status != 0:
        raise DDAError(status, last_error())


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _prec_of(t: torch.Tensor) -> int:
    if t.dtype == torch.complex128:
        return C128
    if t.dtype == torch.complex64:
        return C64
    raise TypeError(f"box fields are complex64 or complex128, got {t.dtype}")


def workspace_size(l, m, n, dx, k, n_materials=1, max_rhs=1, krylov_m=0,
                   precisions=PLAN_C128 | PLAN_C64, precond2=0, circulant="chan",
                   voxel_eps=False, rhs_chunk=0, krylov_c64=False, sstep=0) -> int:
    d = PlanDesc(l, m, n, dx, k, n_materials, max_rhs, krylov_m, precisions,
                 _precond2_code(precond2, (l, m, n)), CIRCULANTS[circulant], int(bool(voxel_eps)),
                 int(rhs_chunk), int(bool(krylov_c64)), int(sstep))
    return int(_lib.dda_workspace_size(ctypes.byref(d)))


@dataclass
class SolveResult:
    x: torch.Tensor
    iters: list
    cycles: list
    converged: list
    rel_resid: list
    status: int
    reorth: list
    history: list = None     # per RHS: relative residual after each inner iteration
    graph: bool = False      # the solve ran as one CUDA graph launch
    ms: float = 0.0          # wall time of the library call


def _result(x, stats, st, hist=None, cap=0):
    h = None
    if hist is not None:
        h = [np.array(hist[r * cap: r * cap + s.history_len]) for r, s in enumerate(stats)]
    return SolveResult(x, [s.iters for s in stats], [s.cycles for s in stats],
                       [bool(s.converged) for s in stats], [s.rel_resid for s in stats], st,
                       [s.reorth for s in stats], h, bool(stats[0].graph) if len(stats) else False,
                       float(stats[0].ms) if len(stats) else 0.0)


class Plan:
    """A DDA problem on one box: geometry, materials, wavenumber, workspace."""

    def __init__(self, mat: torch.Tensor, eps, dx: float, k: float, max_rhs: int = 1,
                 krylov_m: int = 0, precisions: int = PLAN_C128 | PLAN_C64,
                 precond2=False, circulant: str = "chan", voxel_eps: torch.Tensor | None = None,
                 rhs_chunk: int = 0, krylov_c64: bool = False, sstep: int = 0):
        """mat: (n, m, l) uint8 material per voxel (0 air); eps: permittivity of
        materials 1..K; voxel_eps: optional (n, m, l) complex128 permittivity of
        every voxel (dda_set_voxel_eps), which then overrides the table on
        scatterer voxels (the table still gives alpha_tilde); rhs_chunk: right-hand
        sides per pass through the FFT scratch (0: all of max_rhs); krylov_c64:
        Krylov basis in complex64 (complex64 cycles only, half the memory);
        sstep: block size reserved for the s-step GMRES (solve method=2)."""
        if mat.dtype != torch.uint8 or not mat.is_cuda or mat.dim() != 3:
            raise TypeError("mat must be a (n, m, l) uint8 CUDA tensor")
        self.mat = mat.contiguous()
        n, m, l = self.mat.shape
        self.shape = (l, m, n)
        eps = [complex(e) for e in eps]
        self.desc = PlanDesc(l, m, n, float(dx), float(k), len(eps), int(max_rhs), int(krylov_m),
                             int(precisions), _precond2_code(precond2, (l, m, n)),
                             CIRCULANTS[circulant], int(voxel_eps is not None), int(rhs_chunk),
                             int(bool(krylov_c64)), int(sstep))
        size = int(_lib.dda_workspace_size(ctypes.byref(self.desc)))
        if size == 0:
            raise DDAError(1, last_error())
        self.work = torch.empty(size, dtype=torch.uint8, device=self.mat.device)
        heps = (ctypes.c_double * (2 * len(eps)))(*[v for e in eps for v in (e.real, e.imag)])
        h = ctypes.c_void_p()
        _check(_lib.dda_plan_create(ctypes.byref(h), ctypes.byref(self.desc), _ptr(self.mat), heps,
                                    _ptr(self.work), size, _stream()))
        self._h = h
        self.nrhs = 0
        self.voxel_eps = None
        if voxel_eps is not None:
            self.set_voxel_eps(voxel_eps)

    def set_voxel_eps(self, eps: torch.Tensor | None):
        """dda_set_voxel_eps: (n, m, l) complex128 permittivity per voxel, or None."""
        if eps is None:
            _check(_lib.dda_set_voxel_eps(self._h, None, _stream()))
            self.voxel_eps = None
            return
        n, m, l = self.mat.shape
        if tuple(eps.shape) != (n, m, l) or eps.dtype != torch.complex128:
            raise ValueError(f"voxel_eps must be a complex128 tensor of shape {(n, m, l)}")
        if eps.device != self.mat.device:
            raise ValueError("voxel_eps must be on the plan's device")
        self.voxel_eps = eps.contiguous()
        _check(_lib.dda_set_voxel_eps(self._h, _ptr(self.voxel_eps), _stream()))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.dda_plan_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def field_shape(self, nrhs):
        l, m, n = self.shape
        return (nrhs, 3, n, m, l)

    def _field(self, t: torch.Tensor, name: str, dtype=None) -> torch.Tensor:
        """Check a box field against the plan before its pointer reaches a
        kernel: shape (nrhs, 3, n, m, l) with 1 <= nrhs, complex64 or
        complex128 (or exactly `dtype`), on the plan's device; returns it
        contiguous."""
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a tensor")
        if t.dim() != 5 or t.shape[0] < 1 or tuple(t.shape) != self.field_shape(t.shape[0]):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, the plan's box fields are "
                             f"(nrhs, 3, n, m, l) = (nrhs, *{self.field_shape(1)[1:]})")
        if dtype is not None and t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        _prec_of(t)
        if t.device != self.mat.device:
            raise ValueError(f"{name} is on {t.device}, the plan on {self.mat.device}")
        return t.contiguous()

    def _out(self, out: torch.Tensor | None, like: torch.Tensor, name: str = "out",
             may_alias: bool = True) -> torch.Tensor:
        """The output buffer of an apply: a new one like `like`, or the
        caller's, which must match it in shape, dtype and device and be
        contiguous (the library writes through its raw pointer)."""
        if out is None:
            return torch.empty_like(like)
        if not isinstance(out, torch.Tensor):
            raise TypeError(f"{name} must be a tensor")
        if tuple(out.shape) != tuple(like.shape):
            raise ValueError(f"{name} has shape {tuple(out.shape)}, expected {tuple(like.shape)}")
        if out.dtype != like.dtype:
            raise TypeError(f"{name} is {out.dtype}, the input is {like.dtype}")
        if out.device != like.device:
            raise ValueError(f"{name} is on {out.device}, the input on {like.device}")
        if not out.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if not may_alias and out.data_ptr() == like.data_ptr():
            raise ValueError(f"{name} must not be the input buffer")
        return out

    def set_incidence(self, dirs, pols):
        dirs = np.asarray(dirs, dtype=np.float64).reshape(-1, 3)
        pols = np.asarray(pols, dtype=np.float64).reshape(-1, 3)
        arr = (Incidence * len(dirs))()
        for i, (d, e) in enumerate(zip(dirs, pols)):
            arr[i].dir[:] = list(d)
            arr[i].pol[:] = list(e)
        _check(_lib.dda_set_incidence(self._h, len(dirs), arr, _stream()))
        self.nrhs = len(dirs)

    def incident_field(self, nrhs: int | None = None) -> torch.Tensor:
        nrhs = nrhs or self.nrhs
        b = torch.empty(self.field_shape(nrhs), dtype=torch.complex128, device=self.mat.device)
        _check(_lib.dda_incident_field(self._h, nrhs, _ptr(b), _stream()))
        return b

    def matvec(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        x = self._field(x, "x")
        y = self._out(out, x, may_alias=False)
        _check(_lib.dda_matvec(self._h, _prec_of(x), x.shape[0], _ptr(x), _ptr(y), _stream()))
        return y

    def precond_build(self):
        _check(_lib.dda_precond_build(self._h, _stream()))

    def precond_apply(self, v: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        v = self._field(v, "v")
        z = self._out(out, v)
        _check(_lib.dda_precond_apply(self._h, _prec_of(v), v.shape[0], _ptr(v), _ptr(z), _stream()))
        return z

    def precond2_build(self):
        """The paper's 2-level preconditioner (needs a plan made with precond2=True)."""
        _check(_lib.dda_precond2_build(self._h, _stream()))

    def precond2_apply(self, v: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        v = self._field(v, "v")
        z = self._out(out, v)
        _check(_lib.dda_precond2_apply(self._h, _prec_of(v), v.shape[0], _ptr(v), _ptr(z), _stream()))
        return z

    def precond_apply_noalloc(self, v: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        """dda_precond_apply_noalloc: the library's static scratch instead of the workspace."""
        v = self._field(v, "v")
        if out is None:
            raise ValueError("precond_apply_noalloc needs the caller's out buffer")
        out = self._out(out, v)
        _check(_lib.dda_precond_apply_noalloc(self._h, _prec_of(v), v.shape[0], _ptr(v), _ptr(out),
                                              _stream()))
        return out

    def fft3d(self, data: torch.Tensor, inverse: bool = False) -> torch.Tensor:
        """In-place 3-D DFT of (batch, n, m, l) complex arrays."""
        l, m, n = self.shape
        if data.dim() != 4 or tuple(data.shape[1:]) != (n, m, l) or data.shape[0] < 1:
            raise ValueError(f"data has shape {tuple(data.shape)}, expected (batch, {n}, {m}, {l})")
        if not data.is_contiguous():
            raise ValueError("data must be contiguous (the transform is in place)")
        if data.device != self.mat.device:
            raise ValueError(f"data is on {data.device}, the plan on {self.mat.device}")
        nb = data.shape[0]
        _check(_lib.dda_fft3d(self._h, _prec_of(data), nb, _ptr(data), int(inverse), _stream()))
        return data

    def solve(self, b: torch.Tensor | None = None, x0: torch.Tensor | None = None,
              tol: float = 1e-6, max_iters: int = 2000, restart: int = 50, precond: int = 3,
              inner_prec: int = C128, inner_tol: float = 0.0, raise_on_error: bool = True,
              nrhs: int | None = None, reorth_eta: float = 0.5 ** 0.5,
              method: int = 0, history: int = 0, timeout_ms: float = 0.0) -> SolveResult:
        """dda_solve.  method: 0 GMRES, 1 BiCG-Stab, 2 s-step GMRES (the plan's
        sstep); history: entries of residual history kept per right-hand
        side (0: none); timeout_ms: the solve's time limit on the device (0:
        none; a right-hand side stopped by it ends with DDA_ERR_TIMEOUT)."""
        nrhs = nrhs or (b.shape[0] if b is not None else self.nrhs)
        if x0 is None:
            x = torch.zeros(self.field_shape(nrhs), dtype=torch.complex128, device=self.mat.device)
        else:
            x = x0.clone().contiguous()
        hist = (ctypes.c_double * (nrhs * history))() if history > 0 else None
        opts = SolveOpts(tol, max_iters, restart, precond, inner_prec, inner_tol, reorth_eta, method,
                         int(history), int(timeout_ms * 1e6),
                         ctypes.cast(hist, ctypes.POINTER(ctypes.c_double)) if hist is not None
                         else None)
        stats = (RhsStats * nrhs)()
        if b is not None:
            b = self._field(b, "b", torch.complex128)
            if b.shape[0] != nrhs:
                raise ValueError(f"b holds {b.shape[0]} right-hand sides, nrhs is {nrhs}")
        if x0 is not None:
            self._field(x, "x0", torch.complex128)
            if x.shape[0] != nrhs:
                raise ValueError(f"x0 holds {x.shape[0]} right-hand sides, nrhs is {nrhs}")
        bp = _ptr(b) if b is not None else ctypes.c_void_p(0)
        st = _lib.dda_solve(self._h, nrhs, bp, _ptr(x), ctypes.byref(opts), stats, _stream())
        if st != 0 and raise_on_error:
            raise DDAError(st, last_error())
        return _result(x, stats, st, hist, history)

    def adjoint_rhs(self, nrhs: int | None = None) -> torch.Tensor:
        nrhs = nrhs or self.nrhs
        b = torch.empty(self.field_shape(nrhs), dtype=torch.complex128, device=self.mat.device)
        _check(_lib.dda_adjoint_rhs(self._h, nrhs, _ptr(b), _stream()))
        return b

    def ext_gradient_from(self, c: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
        """(nrhs, 2, n, m, l) float64: dC_ext/dRe(eps), dC_ext/dIm(eps) per voxel."""
        c = self._field(c, "c", torch.complex128)
        lam = self._field(lam, "lam", torch.complex128)
        if lam.shape != c.shape:
            raise ValueError("c and lam must hold the same right-hand sides")
        nrhs = c.shape[0]
        l, m, n = self.shape
        g = torch.empty((nrhs, 2, n, m, l), dtype=torch.float64, device=self.mat.device)
        _check(_lib.dda_ext_gradient(self._h, nrhs, _ptr(c), _ptr(lam), _ptr(g), _stream()))
        return g

    def ext_gradient(self, c: torch.Tensor | None = None, **solve_kw):
        """Solve (if c is None), solve the adjoint A lambda = conj(E_inc) with the
        same operator, and return (c, lambda, gradient)."""
        if c is None:
            c = self.solve(**solve_kw).x
        lam = self.solve(b=self.adjoint_rhs(c.shape[0]), **solve_kw).x
        return c, lam, self.ext_gradient_from(c, lam)

    def schedule(self) -> dict:
        s = Schedule()
        _check(_lib.dda_schedule_get(self._h, ctypes.byref(s)))
        return {"rr_z": bool(s.rr_z), "pdl": bool(s.pdl), "graph": bool(s.graph),
                "z_occ": bool(s.z_occ)}

    def set_schedule(self, rr_z: bool = True, pdl: bool = False, graph: bool = True,
                     z_occ: bool = True):
        _check(_lib.dda_schedule_set(self._h, ctypes.byref(Schedule(int(rr_z), int(pdl),
                                                                    int(graph), int(z_occ)))))

    def autotune(self, prec: int = C64, nrhs: int | None = None, reps: int = 10,
                 force: bool = False) -> dict:
        """dda_autotune on the incident field (complex64 or complex128 box
        fields of nrhs right-hand sides); returns the report as a dict."""
        nrhs = nrhs or self.nrhs
        x = self.incident_field(nrhs).to(torch.complex64 if prec == C64 else torch.complex128)
        y = torch.empty_like(x)
        rep = TuneReport()
        _check(_lib.dda_autotune(self._h, prec, nrhs, _ptr(x), _ptr(y), int(reps), int(force),
                                 ctypes.byref(rep), _stream()))
        sched = lambda s: {"rr_z": bool(s.rr_z), "pdl": bool(s.pdl), "graph": bool(s.graph),  # noqa: E731
                           "z_occ": bool(s.z_occ)}
        return {"chosen": sched(rep.chosen), "cached": bool(rep.cached),
                "timed": [(sched(rep.cand[i]), float(rep.ms_per_matvec[i]))
                          for i in range(rep.ncand)]}

    def profile(self, on: bool = True):
        _check(_lib.dda_profile_enable(self._h, int(on)))

    def profile_read(self, reset: bool = True) -> dict:
        """{kernel class: (milliseconds, launches, algorithmic bytes)} since the last read."""
        n = len(PROFILE_NAMES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        byt = (ctypes.c_double * n)()
        _check(_lib.dda_profile_read(self._h, ms, cnt, byt, n, int(reset)))
        return {name: (ms[i], cnt[i], byt[i]) for i, name in enumerate(PROFILE_NAMES)}

    def cross_sections(self, c: torch.Tensor) -> np.ndarray:
        c = self._field(c, "c", torch.complex128)
        nrhs = c.shape[0]
        out = (ctypes.c_double * (3 * nrhs))()
        _check(_lib.dda_cross_sections(self._h, nrhs, _ptr(c), out, _stream()))
        return np.array(out[:], dtype=np.float64).reshape(nrhs, 3)


def solve_many(plans, bs=None, streams=None, tol: float = 1e-6, max_iters: int = 2000,
               restart: int = 50, precond: int = 3, inner_prec: int = C128,
               inner_tol: float = 0.0, reorth_eta: float = 0.5 ** 0.5, method: int = 0,
               raise_on_error: bool = True) -> list:
    """dda_solve_many: the systems of several plans solved concurrently, one
    stream each (created here unless given); returns one SolveResult per plan."""
    n = len(plans)
    cur = torch.cuda.current_stream()
    if streams is None:
        streams = [torch.cuda.Stream(device=p.mat.device) for p in plans]
    xs, stats = [], []
    for p in plans:
        xs.append(torch.zeros(p.field_shape(p.nrhs), dtype=torch.complex128, device=p.mat.device))
        stats.append((RhsStats * p.nrhs)())
    for s in streams:
        s.wait_stream(cur)  # the zeroed x and any b are ready before the solves start
    arr = lambda ptrs: (ctypes.c_void_p * n)(*[ctypes.c_void_p(v) for v in ptrs])
    hp = (ctypes.c_void_p * n)(*[ctypes.c_void_p(p._h.value) for p in plans])
    nr = (ctypes.c_int32 * n)(*[p.nrhs for p in plans])
    bp = arr([b.contiguous().data_ptr() if b is not None else 0 for b in bs]) if bs else None
    xp = arr([x.data_ptr() for x in xs])
    sp = (ctypes.POINTER(RhsStats) * n)(*[ctypes.cast(st, ctypes.POINTER(RhsStats)) for st in stats])
    strp = arr([s.cuda_stream for s in streams])
    opts = SolveOpts(tol, max_iters, restart, precond, inner_prec, inner_tol, reorth_eta, method,
                     0, 0, None)
    st = _lib.dda_solve_many(n, hp, nr, bp, xp, ctypes.byref(opts), sp, strp)
    for s in streams:
        cur.wait_stream(s)
    if st != 0 and raise_on_error:
        raise DDAError(st, last_error())
    return [_result(x, sv, st) for x, sv in zip(xs, stats)]


class _Extinction(torch.autograd.Function):
    """C_ext of each incident wave as a differentiable function of the
    permittivities: one per material (eps of shape (K,)) or one per voxel (eps
    of shape (n, m, l), dda_set_voxel_eps).  Forward: plan, preconditioner,
    solve, C_ext.  Backward: the adjoint solve A lambda = conj(E_inc) with the
    same operator (A = A^T), the per-voxel gradient dC_ext/d eps_j
    (dda_ext_gradient), weighted by the incoming gradient of each wave and
    summed over waves on the device; per material it is then summed over the
    material's voxels (one index_add).  For a real output and a complex input
    the gradient follows PyTorch's convention: dC/dRe(eps) + i dC/dIm(eps)."""

    @staticmethod
    def forward(ctx, eps, geometry, solve_kw, plan_factory):
        mat, dx, k, dirs, pols = geometry
        per_voxel = eps.dim() == 3
        if per_voxel:
            e = eps.detach().to(mat.device, torch.complex128).contiguous()
            sel = mat > 0
            # alpha_tilde (air rows, preconditioner) from the scatterer's mean permittivity
            table = [complex(e[sel].mean().item()) if bool(sel.any()) else complex(e.mean().item())]
        else:
            table = [complex(v) for v in eps.detach().cpu().tolist()]
        pc = solve_kw.get("precond", 3)
        extra = {"voxel_eps": e} if per_voxel else {}
        plan = plan_factory(mat, table, dx, k, len(dirs), max(7, solve_kw.get("restart", 50)),
                            pc == 2, **extra)
        plan.set_incidence(dirs, pols)
        if pc == 3:
            plan.precond_build()
        elif pc == 2:
            plan.precond2_build()
        c = plan.solve(**solve_kw).x
        cext = torch.as_tensor(plan.cross_sections(c)[:, 0], dtype=torch.float64)
        ctx.state = (plan, c, solve_kw, mat, len(table), eps.device, per_voxel)
        return cext

    @staticmethod
    def backward(ctx, grad_out):
        plan, c, solve_kw, mat, K, dev, per_voxel = ctx.state
        lam = plan.solve(b=plan.adjoint_rhs(c.shape[0]), **solve_kw).x
        g = plan.ext_gradient_from(c, lam)  # (nrhs, 2, n, m, l)
        w = grad_out.to(g.device, g.dtype).view(-1, 1, 1, 1, 1)
        gsum = (w * g).sum(dim=0)  # (2, n, m, l): dL/dRe eps_j, dL/dIm eps_j
        gc = torch.complex(gsum[0], gsum[1])
        if per_voxel:
            return gc.to(dev), None, None, None
        idx = mat.reshape(-1).to(gc.device, torch.long)
        per_mat = torch.zeros(K + 1, dtype=torch.complex128, device=gc.device)
        per_mat.index_add_(0, idx, gc.reshape(-1))
        return per_mat[1:].to(dev), None, None, None


def _default_plan_factory(mat, eps, dx, k, nrhs, krylov_m, precond2, voxel_eps=None):
    return Plan(mat, eps, dx, k, max_rhs=nrhs, krylov_m=krylov_m, precond2=precond2,
                voxel_eps=voxel_eps)


def extinction(eps: torch.Tensor, mat: torch.Tensor, dx: float, k: float, dirs, pols,
               plan_factory=_default_plan_factory, **solve_kw) -> torch.Tensor:
    """C_ext per incident wave (float64, shape (nrhs,)), differentiable with
    respect to eps (complex128): one permittivity per material 1..K (shape
    (K,)), or one per voxel (shape (n, m, l); entries on air voxels are
    ignored and get zero gradient).  The gradient is the adjoint one of
    dda_ext_gradient."""
    return _Extinction.apply(eps, (mat, dx, k, list(dirs), list(pols)), dict(solve_kw),
                             plan_factory)
