"""GB300 SAIT: sparse approximate inverses of triangular factors (arXiv 2106.12836).

A thin ctypes binding over ``libsait.so`` whose functions carry the names of
the C ABI in ``include/sait.h``.  It only marshals arguments: every step of
the computation runs in the library's CUDA kernels.  Device buffers are torch
tensors (int32 row pointers / columns, float64 values and vectors); the
library runs on the stream of the context, by default torch's current stream.

The library must have been built (``paper_2106_12836_gb300.build.build()``);
importing this package on a machine where it is missing raises at once.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from . import build as _build

__all__ = [
    "SaitError", "Context", "Mat", "Prec", "Info", "DROP", "DTYPE",
    "sait_ctx_create", "sait_ctx_destroy", "sait_status_string", "sait_ctx_last_error",
    "sait_mat_create_csr", "sait_mat_destroy", "sait_mat_info", "sait_mat_export_csr",
    "sait_mat_set_store", "sait_ilu0", "sait_iluk", "sait_build", "sait_spmv", "sait_apply",
    "sait_prec_create_sait", "sait_prec_create_ilu", "sait_prec_levels", "sait_prec_apply",
    "sait_prec_destroy", "sait_gmres", "sait_bicgstab", "sait_ctx_set_timing", "sait_ctx_stats",
    "sait_apply_static", "APPLY_STATIC_MAX_N", "sait_spmm", "sait_apply_multi", "sait_mat_transpose",
    "sait_outer_on_pattern", "sait_bicgstab_batched", "sait_bicgstab_multi", "BatchInfo", "Stats",
    "TIMERS", "lib_path", "EXPORTS", "sait_lobpcg", "sait_pcg", "sait_prec_create_jacobi", "sait_ilut",
    "sait_mat_autotune", "sait_batch_autotune", "sait_ctx_set_batch_tile", "sait_tune_params",
    "sait_ctx_set_wait_limit", "sait_ctx_set_timing_groups", "sait_ctx_set_device_loop", "SOLVER", "ParamReport",
]

DROP = {"none": 0, "abs": 1, "rowrel": 2, "pattern": 3, "hybrid": 4}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2, "f32x64": 3, "bf16x64": 4}
LOWER, UPPER = 0, 1

# Every entry point declared in include/sait.h.
EXPORTS = [
    "sait_ctx_create", "sait_ctx_destroy", "sait_status_string", "sait_ctx_last_error",
    "sait_mat_create_csr", "sait_mat_destroy", "sait_mat_info", "sait_mat_export_csr",
    "sait_mat_set_store", "sait_ilu0", "sait_iluk", "sait_build", "sait_spmv", "sait_apply",
    "sait_prec_create_sait", "sait_prec_create_ilu", "sait_prec_levels", "sait_prec_apply",
    "sait_prec_destroy", "sait_gmres", "sait_bicgstab", "sait_ctx_set_timing", "sait_ctx_stats",
    "sait_apply_static", "sait_spmm", "sait_apply_multi", "sait_mat_transpose", "sait_outer_on_pattern",
    "sait_bicgstab_batched", "sait_bicgstab_multi", "sait_lobpcg", "sait_pcg", "sait_prec_create_jacobi", "sait_ilut",
    "sait_mat_autotune", "sait_batch_autotune", "sait_ctx_set_batch_tile", "sait_tune_params",
    "sait_ctx_set_wait_limit", "sait_ctx_set_timing_groups", "sait_ctx_set_device_loop",
]
SOLVER = {"gmres": 0, "bicgstab": 1, "pcg": 2}
PARAM_MAX = 16  # SAIT_PARAM_MAX in include/sait.h
APPLY_STATIC_MAX_N = 2097152  # SAIT_APPLY_STATIC_MAX_N in include/sait.h
TIMERS = ["apply", "spmv", "ortho", "build", "ilu", "trisolve"]


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class _Drop(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_int32), ("tau", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double * 6), ("calls", C.c_int64 * 6)]

    def as_dict(self):
        return {"launches": int(self.launches),
                **{t: {"ms": float(self.ms[i]), "calls": int(self.calls[i])}
                   for i, t in enumerate(TIMERS)}}


class BatchInfo(C.Structure):
    _fields_ = [("nsys", C.c_int32), ("converged", C.c_int32), ("max_iters", C.c_int32),
                ("graph_replays", C.c_int32), ("max_rel_resid", C.c_double), ("device_loop", C.c_int32),
                ("graph_launches", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneReport(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("chosen", C.c_int32), ("format", C.c_int32 * 6),
                ("lanes", C.c_int32 * 6), ("us", C.c_float * 6)]

    def as_dict(self):
        return {"chosen": {"format": ("csr", "sell32")[self.format[self.chosen]], "lanes": self.lanes[self.chosen]},
                "candidates": [{"format": ("csr", "sell32")[self.format[i]], "lanes": self.lanes[i],
                                "us": round(self.us[i], 2)} for i in range(self.ncand)]}


class _Param(C.Structure):
    _fields_ = [("m_terms", C.c_int32), ("pad", C.c_int32), ("drop", _Drop)]


class ParamReport(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("chosen", C.c_int32), ("status", C.c_int32 * PARAM_MAX),
                ("iters", C.c_int32 * PARAM_MAX), ("nnz", C.c_int64 * PARAM_MAX),
                ("build_ms", C.c_float * PARAM_MAX), ("solve_ms", C.c_float * PARAM_MAX),
                ("rel_resid", C.c_double * PARAM_MAX)]

    def as_dict(self, cands=None):
        rows = []
        for i in range(self.ncand):
            r = {"status": self.status[i], "iters": self.iters[i], "nnz": self.nnz[i],
                 "build_ms": round(self.build_ms[i], 3), "solve_ms": round(self.solve_ms[i], 3),
                 "rel_resid": self.rel_resid[i]}
            if cands is not None:
                r["param"] = cands[i]
            rows.append(r)
        return {"chosen": self.chosen, "candidates": rows}


class BatchTuneReport(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("chosen", C.c_int32), ("tile_rows", C.c_int32 * 6), ("us", C.c_float * 6)]

    def as_dict(self):
        return {"chosen_tile_rows": self.tile_rows[self.chosen],
                "candidates": [{"tile_rows": self.tile_rows[i], "us": round(self.us[i], 2)} for i in range(self.ncand)]}


class Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("cycles", C.c_int32), ("reorth_steps", C.c_int32),
                ("pad", C.c_int32), ("rel_resid", C.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "cycles": self.cycles, "reorth_steps": self.reorth_steps,
                "rel_resid": self.rel_resid}


def lib_path() -> str:
    return _build.LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libsait.so not built ({_build.LIB}); run "
                              "paper_2106_12836_gb300.build.build() first")
        lib = C.CDLL(_build.LIB)
        vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sigs = {
            "sait_ctx_create": [C.POINTER(vp), vp],
            "sait_ctx_destroy": [vp],
            "sait_status_string": [C.c_int],
            "sait_ctx_last_error": [vp],
            "sait_mat_create_csr": [vp, C.POINTER(_Csr), C.POINTER(vp)],
            "sait_mat_destroy": [vp],
            "sait_mat_info": [vp, C.POINTER(i64), C.POINTER(i64)],
            "sait_mat_export_csr": [vp, vp, vp, vp, vp],
            "sait_mat_set_store": [vp, vp, C.c_int],
            "sait_ilu0": [vp, C.POINTER(_Csr), C.POINTER(vp), C.POINTER(vp)],
            "sait_iluk": [vp, C.POINTER(_Csr), i32, C.POINTER(vp), C.POINTER(vp)],
            "sait_build": [vp, vp, C.c_int, i32, _Drop, C.c_int, C.POINTER(vp)],
            "sait_spmv": [vp, vp, vp, vp],
            "sait_apply": [vp, vp, vp, vp, vp],
            "sait_prec_create_sait": [vp, vp, vp, C.POINTER(vp)],
            "sait_prec_create_ilu": [vp, vp, vp, C.POINTER(vp)],
            "sait_prec_levels": [vp, C.POINTER(i32), C.POINTER(i32)],
            "sait_prec_apply": [vp, vp, vp, vp],
            "sait_prec_destroy": [vp],
            "sait_gmres": [vp, vp, vp, vp, vp, i32, d, i32, C.POINTER(Info)],
            "sait_bicgstab": [vp, vp, vp, vp, vp, d, i32, C.POINTER(Info)],
            "sait_ctx_set_timing": [vp, C.c_int],
            "sait_ctx_set_wait_limit": [vp, i64],
            "sait_ctx_set_device_loop": [vp, i32],
            "sait_ctx_set_timing_groups": [vp, C.c_uint32, i32],
            "sait_ctx_stats": [vp, C.POINTER(Stats), C.c_int],
            "sait_apply_static": [vp, vp, vp, vp, vp],
            "sait_spmm": [vp, vp, i32, vp, i64, vp, i64],
            "sait_apply_multi": [vp, vp, vp, i32, vp, i64, vp, i64],
            "sait_mat_transpose": [vp, vp, C.POINTER(vp)],
            "sait_outer_on_pattern": [vp, vp, d, vp, vp, vp],
            "sait_bicgstab_batched": [vp, vp, vp, i32, vp, vp, vp, d, i32, C.POINTER(BatchInfo), vp, vp],
            "sait_bicgstab_multi": [vp, vp, vp, i32, vp, vp, d, i32, C.POINTER(BatchInfo), vp, vp],
            "sait_lobpcg": [vp, vp, vp, i32, vp, vp, d, i32, C.POINTER(Info)],
            "sait_pcg": [vp, vp, vp, vp, vp, d, i32, C.POINTER(Info)],
            "sait_prec_create_jacobi": [vp, vp, vp, i32, C.POINTER(vp)],
            "sait_ilut": [vp, C.POINTER(_Csr), d, i32, C.POINTER(vp), C.POINTER(vp)],
            "sait_mat_autotune": [vp, vp, C.POINTER(TuneReport)],
            "sait_batch_autotune": [vp, i64, i32, vp, C.POINTER(BatchTuneReport)],
            "sait_ctx_set_batch_tile": [vp, i64],
            "sait_tune_params": [vp, vp, vp, vp, vp, vp, C.c_int, i32, d, i32, i32, C.POINTER(_Param), C.c_int,
                                 i32, C.POINTER(ParamReport)],
        }
        for name, args in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        lib.sait_status_string.restype = C.c_char_p
        lib.sait_ctx_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


class SaitError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


def _check(ctx, st: int, what: str):
    if st != 0:
        detail = _L().sait_ctx_last_error(ctx.h if ctx is not None else None)
        detail = detail.decode() if detail else ""
        raise SaitError(st, f"{what}: {sait_status_string(st)}; {detail}")


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _ptr_any(t: torch.Tensor):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return t.data_ptr() if t.numel() else None


def _vec(t: torch.Tensor, n: int, name: str) -> torch.Tensor:
    if t.dtype != torch.float64 or t.numel() != n or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor of {n} entries")
    return t


class Context:
    """Owns a sait_ctx bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = None
        self.h = sait_ctx_create(self.stream.cuda_stream)

    def close(self):
        if self.h is not None:
            sait_ctx_destroy(self)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Mat:
    """A library-owned CSR matrix (sait_mat)."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        self.n, self.nnz = sait_mat_info(self)

    def export(self):
        return sait_mat_export_csr(self.ctx, self)

    def close(self):
        if self.h is not None:
            sait_mat_destroy(self)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Prec:
    """A preconditioner object (sait_prec); keeps its matrices alive."""

    def __init__(self, ctx: Context, h, mats):
        self.ctx, self.h, self._mats = ctx, h, mats
        self.n = mats[0].n

    def close(self):
        if self.h is not None:
            sait_prec_destroy(self)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _csr(n: int, rp: torch.Tensor, ci: torch.Tensor, va: torch.Tensor) -> _Csr:
    if rp.dtype != torch.int32 or ci.dtype != torch.int32 or va.dtype != torch.float64:
        raise ValueError("CSR arrays must be int32 row_ptr, int32 col, float64 val")
    if rp.numel() != n + 1 or ci.numel() != va.numel():
        raise ValueError("CSR array sizes do not match")
    return _Csr(n, va.numel(), _ptr(rp), _ptr(ci) if ci.numel() else None,
                _ptr(va) if va.numel() else None)


# ---- C ABI, one Python function per entry point -------------------------------
def sait_status_string(st: int) -> str:
    return _L().sait_status_string(st).decode()


def sait_ctx_create(stream_handle: int):
    h = C.c_void_p()
    st = _L().sait_ctx_create(C.byref(h), C.c_void_p(stream_handle))
    if st:
        raise SaitError(st, "sait_ctx_create: " + sait_status_string(st))
    return h


def sait_ctx_destroy(ctx: Context):
    _check(None, _L().sait_ctx_destroy(ctx.h), "sait_ctx_destroy")


def sait_ctx_set_timing(ctx: Context, enable: bool):
    _check(ctx, _L().sait_ctx_set_timing(ctx.h, int(bool(enable))), "sait_ctx_set_timing")


def sait_ctx_set_timing_groups(ctx: Context, groups=None, every: int = 1):
    """Time only the named groups (names of TIMERS; None: all of them), one call
    in `every` of each."""
    mask = 0xFFFFFFFF if groups is None else sum(1 << TIMERS.index(g) for g in groups)
    _check(ctx, _L().sait_ctx_set_timing_groups(ctx.h, mask, int(every)), "sait_ctx_set_timing_groups")


def sait_ctx_set_wait_limit(ctx: Context, polls: int = 0):
    """Polls a device-side dependency wait makes before giving up (0: the default)."""
    _check(ctx, _L().sait_ctx_set_wait_limit(ctx.h, int(polls)), "sait_ctx_set_wait_limit")


def sait_ctx_set_device_loop(ctx: Context, on: bool = True):
    """Batched solvers: iterate inside a WHILE graph node (True) or replay the
    iteration graph from the host (False; what kernel profilers can see)."""
    _check(ctx, _L().sait_ctx_set_device_loop(ctx.h, int(bool(on))), "sait_ctx_set_device_loop")


def sait_ctx_stats(ctx: Context, reset: bool = False) -> Stats:
    st = Stats()
    _check(ctx, _L().sait_ctx_stats(ctx.h, C.byref(st), int(bool(reset))), "sait_ctx_stats")
    return st


def sait_ctx_last_error(ctx: Context) -> str:
    return _L().sait_ctx_last_error(ctx.h).decode()


def sait_mat_create_csr(ctx: Context, n: int, rp, ci, va) -> Mat:
    A = _csr(n, rp, ci, va)
    h = C.c_void_p()
    _check(ctx, _L().sait_mat_create_csr(ctx.h, C.byref(A), C.byref(h)), "sait_mat_create_csr")
    return Mat(ctx, h)


def sait_mat_destroy(M: Mat):
    _check(None, _L().sait_mat_destroy(M.h), "sait_mat_destroy")


def sait_mat_info(M: Mat):
    n, nnz = C.c_int64(), C.c_int64()
    _check(None, _L().sait_mat_info(M.h, C.byref(n), C.byref(nnz)), "sait_mat_info")
    return int(n.value), int(nnz.value)


def sait_mat_export_csr(ctx: Context, M: Mat):
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.empty(M.n + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(max(M.nnz, 1), dtype=torch.int32, device=dev)
    va = torch.empty(max(M.nnz, 1), dtype=torch.float64, device=dev)
    _check(ctx, _L().sait_mat_export_csr(ctx.h, M.h, _ptr(rp), _ptr(ci), _ptr(va)),
           "sait_mat_export_csr")
    return rp, ci[:M.nnz], va[:M.nnz]


def sait_mat_set_store(ctx: Context, M: Mat, store: str):
    _check(ctx, _L().sait_mat_set_store(ctx.h, M.h, DTYPE[store]), "sait_mat_set_store")


def sait_ilu0(ctx: Context, n: int, rp, ci, va):
    A = _csr(n, rp, ci, va)
    hl, hu = C.c_void_p(), C.c_void_p()
    _check(ctx, _L().sait_ilu0(ctx.h, C.byref(A), C.byref(hl), C.byref(hu)), "sait_ilu0")
    return Mat(ctx, hl), Mat(ctx, hu)


def sait_iluk(ctx: Context, n: int, rp, ci, va, level: int):
    """Level-of-fill ILU(level) factors, level 0 or 1 (Saad, Algorithm 10.5): (L, U) as sait_ilu0."""
    A = _csr(n, rp, ci, va)
    hl, hu = C.c_void_p(), C.c_void_p()
    _check(ctx, _L().sait_iluk(ctx.h, C.byref(A), int(level), C.byref(hl), C.byref(hu)), "sait_iluk")
    return Mat(ctx, hl), Mat(ctx, hu)


def sait_ilut(ctx: Context, n: int, rp, ci, va, tau: float, lfil: int):
    """ILUT(tau, lfil) factors (Saad, Algorithm 10.6): (L, U) as sait_ilu0."""
    A = _csr(n, rp, ci, va)
    hl, hu = C.c_void_p(), C.c_void_p()
    _check(ctx, _L().sait_ilut(ctx.h, C.byref(A), float(tau), int(lfil), C.byref(hl), C.byref(hu)), "sait_ilut")
    return Mat(ctx, hl), Mat(ctx, hu)


def sait_build(ctx: Context, T: Mat, lower: bool, m_terms: int, drop: str = "rowrel",
               tau: float = 0.0, p: int = 0, store: str = "f64") -> Mat:
    h = C.c_void_p()
    d = _Drop(DROP[drop], int(p), float(tau))
    _check(ctx, _L().sait_build(ctx.h, T.h, LOWER if lower else UPPER, int(m_terms), d,
                                DTYPE[store], C.byref(h)), "sait_build")
    return Mat(ctx, h)


def sait_spmv(ctx: Context, A: Mat, x: torch.Tensor, y: torch.Tensor | None = None):
    _vec(x, A.n, "x")
    y = torch.empty_like(x) if y is None else _vec(y, A.n, "y")
    _check(ctx, _L().sait_spmv(ctx.h, A.h, _ptr(x), _ptr(y)), "sait_spmv")
    return y


def sait_apply(ctx: Context, ML: Mat, MU: Mat, r: torch.Tensor, z: torch.Tensor | None = None):
    _vec(r, ML.n, "r")
    z = torch.empty_like(r) if z is None else _vec(z, ML.n, "z")
    _check(ctx, _L().sait_apply(ctx.h, ML.h, MU.h, _ptr(r), _ptr(z)), "sait_apply")
    return z


def sait_apply_static(ML: Mat, MU: Mat, r: torch.Tensor, z: torch.Tensor,
                      stream: torch.cuda.Stream | None = None) -> int:
    """z = M_U (M_L r) without any allocation by the library (see include/sait.h).

    For callers that cannot allow device allocations at apply time
    (allocator-free loops, runtimes that own all device memory): the
    intermediate vector lives in a fixed array inside the library, shared by
    all calls on a device, so calls that overlap on the GPU race.  n must not exceed
    APPLY_STATIC_MAX_N.  Returns the status code (0 = ok) instead of raising,
    since no context records a message.
    """
    _vec(r, ML.n, "r")
    _vec(z, ML.n, "z")
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(_L().sait_apply_static(ML.h, MU.h, _ptr(r), _ptr(z), C.c_void_p(s.cuda_stream)))


def _block(t: torch.Tensor, n: int, name: str) -> torch.Tensor:
    if t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2 or t.shape[0] != n or t.stride(1) != 1:
        raise ValueError(f"{name}: expected a float64 CUDA block of {n} rows with unit column stride")
    return t


def sait_spmm(ctx: Context, A: Mat, X: torch.Tensor, Y: torch.Tensor | None = None) -> torch.Tensor:
    """Y = A X for a row-major n x k block."""
    _block(X, A.n, "X")
    Y = torch.empty_like(X) if Y is None else _block(Y, A.n, "Y")
    _check(ctx, _L().sait_spmm(ctx.h, A.h, X.shape[1], _ptr_any(X), X.stride(0), _ptr_any(Y), Y.stride(0)),
           "sait_spmm")
    return Y


def sait_apply_multi(ctx: Context, ML: Mat, MU: Mat, R: torch.Tensor, Z: torch.Tensor | None = None):
    """Z = M_U (M_L R) for a row-major n x k block."""
    _block(R, ML.n, "R")
    Z = torch.empty_like(R) if Z is None else _block(Z, ML.n, "Z")
    _check(ctx, _L().sait_apply_multi(ctx.h, ML.h, MU.h, R.shape[1], _ptr_any(R), R.stride(0), _ptr_any(Z),
                                      Z.stride(0)), "sait_apply_multi")
    return Z


def sait_mat_transpose(ctx: Context, M: Mat) -> Mat:
    h = C.c_void_p()
    _check(ctx, _L().sait_mat_transpose(ctx.h, M.h, C.byref(h)), "sait_mat_transpose")
    return Mat(ctx, h)


def sait_outer_on_pattern(ctx: Context, A: Mat, alpha: float, u: torch.Tensor, v: torch.Tensor,
                          out: torch.Tensor | None = None) -> torch.Tensor:
    """out[e] = alpha * u[row(e)] * v[col(e)] over A's stored entries (CSR order)."""
    _vec(u, A.n, "u")
    _vec(v, A.n, "v")
    out = torch.empty(A.nnz, dtype=torch.float64, device=u.device) if out is None else out
    _check(ctx, _L().sait_outer_on_pattern(ctx.h, A.h, float(alpha), _ptr(u), _ptr(v), _ptr_any(out)),
           "sait_outer_on_pattern")
    return out


def sait_prec_create_sait(ctx: Context, ML: Mat, MU: Mat) -> Prec:
    h = C.c_void_p()
    _check(ctx, _L().sait_prec_create_sait(ctx.h, ML.h, MU.h, C.byref(h)), "sait_prec_create_sait")
    return Prec(ctx, h, (ML, MU))


def sait_prec_create_ilu(ctx: Context, L: Mat, U: Mat) -> Prec:
    h = C.c_void_p()
    _check(ctx, _L().sait_prec_create_ilu(ctx.h, L.h, U.h, C.byref(h)), "sait_prec_create_ilu")
    return Prec(ctx, h, (L, U))


def sait_prec_create_jacobi(ctx: Context, L: Mat, U: Mat, sweeps: int) -> Prec:
    h = C.c_void_p()
    _check(ctx, _L().sait_prec_create_jacobi(ctx.h, L.h, U.h, int(sweeps), C.byref(h)),
           "sait_prec_create_jacobi")
    return Prec(ctx, h, [L, U])


def sait_prec_levels(P: Prec):
    a, b = C.c_int32(), C.c_int32()
    _check(None, _L().sait_prec_levels(P.h, C.byref(a), C.byref(b)), "sait_prec_levels")
    return int(a.value), int(b.value)


def sait_prec_apply(ctx: Context, P: Prec, r: torch.Tensor, z: torch.Tensor | None = None):
    _vec(r, P.n, "r")
    z = torch.empty_like(r) if z is None else _vec(z, P.n, "z")
    _check(ctx, _L().sait_prec_apply(ctx.h, P.h, _ptr(r), _ptr(z)), "sait_prec_apply")
    return z


def sait_prec_destroy(P: Prec):
    _check(None, _L().sait_prec_destroy(P.h), "sait_prec_destroy")


def sait_gmres(ctx: Context, A: Mat, P: Prec | None, b: torch.Tensor, x: torch.Tensor | None = None,
               restart: int = 30, tol: float = 1e-8, maxit: int = 10000, check: bool = True):
    _vec(b, A.n, "b")
    x = torch.zeros_like(b) if x is None else _vec(x, A.n, "x")
    info = Info()
    st = _L().sait_gmres(ctx.h, A.h, P.h if P is not None else None, _ptr(b), _ptr(x),
                         int(restart), float(tol), int(maxit), C.byref(info))
    if check:
        _check(ctx, st, "sait_gmres")
    return x, info, st


def sait_bicgstab(ctx: Context, A: Mat, P: Prec | None, b: torch.Tensor,
                  x: torch.Tensor | None = None, tol: float = 1e-8, maxit: int = 10000,
                  check: bool = True):
    _vec(b, A.n, "b")
    x = torch.zeros_like(b) if x is None else _vec(x, A.n, "x")
    info = Info()
    st = _L().sait_bicgstab(ctx.h, A.h, P.h if P is not None else None, _ptr(b), _ptr(x),
                            float(tol), int(maxit), C.byref(info))
    if check:
        _check(ctx, st, "sait_bicgstab")
    return x, info, st


def sait_bicgstab_batched(ctx: Context, A: Mat, P: Prec | None, sys_ptr: torch.Tensor, b: torch.Tensor,
                          x: torch.Tensor | None = None, tol: float = 1e-8, maxit: int = 10000,
                          check: bool = True):
    """BiCGSTAB on the independent diagonal blocks of A (rows sys_ptr[s]..sys_ptr[s+1]).

    Returns (x, BatchInfo, status, per-system relative residuals, per-system iterations).
    """
    if sys_ptr.dtype != torch.int64 or not sys_ptr.is_cuda:
        raise ValueError("sys_ptr: int64 CUDA tensor of nsys + 1 offsets")
    nsys = sys_ptr.numel() - 1
    _vec(b, A.n, "b")
    x = torch.zeros_like(b) if x is None else _vec(x, A.n, "x")
    rr = torch.empty(nsys, dtype=torch.float64, device=b.device)
    its = torch.empty(nsys, dtype=torch.int32, device=b.device)
    info = BatchInfo()
    st = _L().sait_bicgstab_batched(ctx.h, A.h, P.h if P is not None else None, nsys, _ptr(sys_ptr), _ptr(b),
                                    _ptr(x), float(tol), int(maxit), C.byref(info), _ptr(rr), _ptr(its))
    if check:
        _check(ctx, st, "sait_bicgstab_batched")
    return x, info, st, rr, its


def sait_bicgstab_multi(ctx: Context, A: Mat, P: Prec | None, B: torch.Tensor, X: torch.Tensor | None = None,
                        tol: float = 1e-8, maxit: int = 10000, check: bool = True):
    """BiCGSTAB for the k columns of the row-major n x k block B at once.

    Returns (X, BatchInfo, status, per-column relative residuals, per-column iterations).
    """
    if B.dim() != 2 or not B.is_contiguous():
        raise ValueError("B: contiguous row-major n x k block")
    _block(B, A.n, "B")
    k = B.shape[1]
    X = torch.zeros_like(B) if X is None else _block(X, A.n, "X")
    rr = torch.empty(k, dtype=torch.float64, device=B.device)
    its = torch.empty(k, dtype=torch.int32, device=B.device)
    info = BatchInfo()
    st = _L().sait_bicgstab_multi(ctx.h, A.h, P.h if P is not None else None, k, _ptr_any(B), _ptr_any(X),
                                  float(tol), int(maxit), C.byref(info), _ptr(rr), _ptr(its))
    if check:
        _check(ctx, st, "sait_bicgstab_multi")
    return X, info, st, rr, its


def sait_lobpcg(ctx: Context, A: Mat, P: Prec | None, X: torch.Tensor, tol: float = 1e-8, maxit: int = 500,
                check: bool = True):
    """k smallest eigenpairs of SPD A by LOBPCG; X (n x k, row-major) is the initial block.

    Returns (lambda, X, info, status); X is overwritten with the eigenvectors.
    """
    if X.dim() != 2 or not X.is_contiguous():
        raise ValueError("X: contiguous row-major n x k block")
    _block(X, A.n, "X")
    lam = torch.empty(X.shape[1], dtype=torch.float64, device=X.device)
    info = Info()
    st = _L().sait_lobpcg(ctx.h, A.h, P.h if P is not None else None, X.shape[1], _ptr_any(X), _ptr(lam),
                          float(tol), int(maxit), C.byref(info))
    if check:
        _check(ctx, st, "sait_lobpcg")
    return lam, X, info, st


def sait_pcg(ctx: Context, A: Mat, P: Prec | None, b: torch.Tensor, x: torch.Tensor | None = None,
             tol: float = 1e-10, maxit: int = 10000, check: bool = True):
    """Preconditioned CG (the paper's solver).  Returns (x, info, status)."""
    _vec(b, A.n, "b")
    x = torch.zeros_like(b) if x is None else _vec(x, A.n, "x")
    info = Info()
    st = _L().sait_pcg(ctx.h, A.h, P.h if P is not None else None, _ptr(b), _ptr(x), float(tol), int(maxit),
                       C.byref(info))
    if check:
        _check(ctx, st, "sait_pcg")
    return x, info, st


def sait_mat_autotune(ctx: Context, M: Mat) -> TuneReport:
    """Time M's product kernels and keep the fastest for later products."""
    r = TuneReport()
    _check(ctx, _L().sait_mat_autotune(ctx.h, M.h, C.byref(r)), "sait_mat_autotune")
    return r


def sait_tune_params(ctx: Context, A: Mat, L: Mat, U: Mat, b: torch.Tensor, candidates,
                     solver: str = "gmres", restart: int = 50, tol: float = 1e-8, maxit: int = 10000,
                     store: str = "f64", count_build: bool = True, x: torch.Tensor | None = None):
    """Time SAIT(L), SAIT(U) + the solve for each candidate and pick the fastest
    (the optimal parameters of Section 3).  candidates: list of dicts with keys
    m_terms, drop (name), tau, p.  Returns (x of the chosen candidate, report)."""
    _vec(b, A.n, "b")
    x = torch.zeros_like(b) if x is None else _vec(x, A.n, "x")
    cands = list(candidates)
    if not 1 <= len(cands) <= PARAM_MAX:
        raise ValueError(f"1..{PARAM_MAX} candidates expected")
    arr = (_Param * len(cands))()
    for i, c in enumerate(cands):
        arr[i].m_terms = int(c["m_terms"])
        arr[i].drop = _Drop(DROP[c.get("drop", "rowrel")], int(c.get("p", 0)), float(c.get("tau", 0.0)))
    r = ParamReport()
    st = _L().sait_tune_params(ctx.h, A.h, L.h, U.h, _ptr(b), _ptr(x), SOLVER[solver], int(restart), float(tol),
                               int(maxit), len(cands), arr, DTYPE[store], int(bool(count_build)), C.byref(r))
    _check(ctx, st, "sait_tune_params")
    return x, r


def sait_batch_autotune(ctx: Context, n: int, sys_ptr: torch.Tensor) -> BatchTuneReport:
    """Choose the batched solver's tile size for this batch (kept in ctx)."""
    if sys_ptr.dtype != torch.int64 or not sys_ptr.is_cuda:
        raise ValueError("sys_ptr: int64 CUDA tensor expected")
    r = BatchTuneReport()
    _check(ctx, _L().sait_batch_autotune(ctx.h, int(n), sys_ptr.numel() - 1, _ptr_any(sys_ptr), C.byref(r)),
           "sait_batch_autotune")
    return r


def sait_ctx_set_batch_tile(ctx: Context, rows: int):
    _check(ctx, _L().sait_ctx_set_batch_tile(ctx.h, int(rows)), "sait_ctx_set_batch_tile")
