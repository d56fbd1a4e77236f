"""ctypes binding of libffsyrk.so (see include/ffsyrk.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Matrices are torch tensors on the current CUDA device holding
uint32 bit patterns (dtype torch.int32 or torch.uint32), row-major with unit
column stride.  If the library is missing this module raises on first use;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libffsyrk.so")

SUCCESS, ERR_INVALID_ARG, ERR_NOT_PRIME, ERR_UNSUPPORTED_P, ERR_ALLOC, ERR_CUDA, ERR_TIMEOUT, \
    ERR_ARCH, ERR_TOO_LARGE = range(9)
LOWER, UPPER = 0, 1
LEAF_AUTO, LEAF_TC_BF16, LEAF_I64, LEAF_I8 = 0, 1, 2, 3
LEVELS_AUTO = -1

_LEAVES = {None: LEAF_AUTO, "auto": LEAF_AUTO, "tc": LEAF_TC_BF16, "bf16": LEAF_TC_BF16,
           "i64": LEAF_I64, "i8": LEAF_I8}

#: every entry point include/ffsyrk.h declares
EXPORTS = ["ffsyrk_options_default", "ffsyrk_plan", "ffsyrk_plan_destroy", "ffsyrk_with_plan",
           "ffsyrk", "ffsyrk_batched", "ffsyrk_sync_status", "ffsyrk_plan_get_info",
           "ffsyrk_plan_set_timing", "ffsyrk_plan_get_timing", "ffsyrk_status_string",
           "ffsyrk_version", "ffsyrk_noalloc", "ffsyrk_leaf_schedule", "ffsyrk_digit_bounds",
           "ffsyrk_digit_base", "ffsyrk_plan_selftest_timeout", "ffsyrk_with_plan_update",
           "ffsyrk_update", "ffsyrkd_with_plan_update", "ffsyrkd_update", "ffsyrkd_factor",
           "ffsyrkbd_with_plan_update", "ffsyrkbd_update", "ffsyrkbd_factor",
           "ffsyrkbd_factor_device", "ffherk_plan", "ffherk_plan_destroy", "ffherk_with_plan",
           "ffherk_sync_status", "ffherk", "ffsyrk_host", "ffsyrk_workspace_query",
           "ffsyrk_test_inject_alloc_failure", "ffsyrk_cache_info", "ffsyrk_probe_pipe",
           "ffsyrk_i8_schedule", "ffsyrk_i8_digit_bounds", "ffsyrk_leaf_schedule_ks",
           "ffsyrk_digit_planes", "ffsyrk_plan_units"]


class FfsyrkError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


class Options(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("tile_ctas", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("winograd", ctypes.c_int32), ("digit_products", ctypes.c_int32),
                ("epilogue_warps", ctypes.c_int32), ("unit_bounds", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("p", ctypes.c_uint32), ("y_form", ctypes.c_int32), ("y_a", ctypes.c_uint32),
                ("y_b", ctypes.c_uint32), ("y_cost", ctypes.c_int32), ("leaf", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("digits", ctypes.c_int32),
                ("chunk_k", ctypes.c_int32 * 9), ("workspace_bytes", ctypes.c_int64),
                ("tile_ctas", ctypes.c_int32), ("autotuned", ctypes.c_int32),
                ("tuned_ms", ctypes.c_float), ("winograd", ctypes.c_int32 * 6),
                ("planes", ctypes.c_int32), ("products", ctypes.c_int32),
                ("epilogue_warps", ctypes.c_int32), ("unit_bounds", ctypes.c_int32)]


class Timing(ctypes.Structure):
    _fields_ = [("prep_ms", ctypes.c_float), ("leaf_ms", ctypes.c_float),
                ("post_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("launches", ctypes.c_int32), ("leaf_launches", ctypes.c_int32),
                ("field_macs", ctypes.c_double), ("tensor_macs", ctypes.c_double),
                ("leaf_tiles", ctypes.c_int32), ("leaf_entries", ctypes.c_int32),
                ("split_tiles", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load libffsyrk.so (raises FileNotFoundError if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise FileNotFoundError(
                    f"{LIB_PATH} is missing: build it with paper_2001_04109_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            i64, u32, vp, i32 = ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int32
            P = ctypes.POINTER
            L.ffsyrk_options_default.argtypes = [P(Options)]
            L.ffsyrk_options_default.restype = None
            L.ffsyrk_plan.argtypes = [P(vp), u32, i64, i64, P(Options)]
            L.ffsyrk_plan_destroy.argtypes = [vp]
            L.ffsyrk_with_plan.argtypes = [vp, i32, i64, i64, u32, vp, i64, vp, i64, vp]
            L.ffsyrk.argtypes = [i32, i64, i64, u32, vp, i64, vp, i64, vp]
            L.ffsyrk_with_plan_update.argtypes = [vp, i32, i64, i64, u32, u32, vp, i64, u32, vp, i64,
                                                  vp]
            L.ffsyrk_update.argtypes = [i32, i64, i64, u32, u32, vp, i64, u32, vp, i64, vp]
            L.ffsyrkd_with_plan_update.argtypes = [vp, i32, i64, i64, u32, u32, vp, i64, P(u32), u32,
                                                   vp, i64, vp]
            L.ffsyrkd_update.argtypes = [i32, i64, i64, u32, u32, vp, i64, P(u32), u32, vp, i64, vp]
            L.ffsyrkd_factor.argtypes = [u32, i64, P(u32), P(i32), P(u32), P(u32)]
            L.ffsyrkd_factor.restype = i32
            L.ffsyrkbd_with_plan_update.argtypes = [vp, i32, i64, i64, u32, u32, vp, i64, P(u32),
                                                    P(u32), u32, vp, i64, vp]
            L.ffsyrkbd_update.argtypes = [i32, i64, i64, u32, u32, vp, i64, P(u32), P(u32), u32, vp,
                                          i64, vp]
            L.ffsyrkbd_factor.argtypes = [u32, i64, P(u32), P(u32), P(i32), P(u32)]
            L.ffsyrkbd_factor.restype = i32
            L.ffsyrkbd_factor_device.argtypes = [u32, i64, P(u32), P(u32), P(i32), P(u32)]
            L.ffsyrkbd_factor_device.restype = i32
            L.ffherk_plan.argtypes = [P(vp), u32, u32, i64, i64, P(Options)]
            L.ffherk_plan_destroy.argtypes = [vp]
            L.ffherk_with_plan.argtypes = [vp, i32, i64, i64, vp, i64, vp, vp, i64, vp]
            L.ffherk_sync_status.argtypes = [vp, vp]
            L.ffherk.argtypes = [i32, i64, i64, u32, u32, vp, i64, vp, vp, i64, vp]
            L.ffsyrk_host.argtypes = [vp, i32, i64, i64, u32, vp, i64, vp, i64, vp]
            L.ffsyrk_host.restype = i32
            L.ffsyrk_workspace_query.argtypes = [u32, i64, i64, P(Options), i32, P(i64), P(i64)]
            L.ffsyrk_workspace_query.restype = i32
            L.ffsyrk_test_inject_alloc_failure.argtypes = [i32, i32]
            L.ffsyrk_test_inject_alloc_failure.restype = i32
            L.ffsyrk_cache_info.argtypes = [P(i32), P(i64)]
            L.ffsyrk_cache_info.restype = i32
            L.ffsyrk_probe_pipe.argtypes = [i32, i64, i32, vp, vp, P(ctypes.c_double)]
            L.ffsyrk_probe_pipe.restype = i32
            L.ffsyrk_plan_units.argtypes = [vp, vp, P(i64), P(i64)]
            L.ffsyrk_plan_units.restype = i32
            for name in ["ffherk_plan", "ffherk_plan_destroy", "ffherk_with_plan",
                         "ffherk_sync_status", "ffherk", "ffsyrk_host", "ffsyrk_workspace_query"]:
                getattr(L, name).restype = i32
            L.ffsyrk_noalloc.argtypes = [i32, i64, i64, u32, vp, i64, vp, i64, vp]
            L.ffsyrk_batched.argtypes = [i32, i64, P(i64), P(i64), u32, P(vp), P(i64), P(vp),
                                         P(i64), vp]
            L.ffsyrk_sync_status.argtypes = [vp, vp]
            L.ffsyrk_plan_get_info.argtypes = [vp, P(PlanInfo)]
            L.ffsyrk_plan_set_timing.argtypes = [vp, i32]
            L.ffsyrk_plan_get_timing.argtypes = [vp, P(Timing)]
            L.ffsyrk_status_string.argtypes = [i32]
            L.ffsyrk_status_string.restype = ctypes.c_char_p
            L.ffsyrk_version.restype = i32
            L.ffsyrk_plan_selftest_timeout.argtypes = [vp, i64, vp]
            L.ffsyrk_plan_selftest_timeout.restype = i32
            L.ffsyrk_leaf_schedule.argtypes = [u32, i32, P(i32), i32]
            L.ffsyrk_leaf_schedule.restype = i32
            L.ffsyrk_digit_bounds.argtypes = [u32, P(i32)]
            L.ffsyrk_digit_bounds.restype = i32
            L.ffsyrk_leaf_schedule_ks.argtypes = [u32, i32, P(i32), i32]
            L.ffsyrk_leaf_schedule_ks.restype = i32
            L.ffsyrk_digit_planes.argtypes = [u32, P(i32), P(u32)]
            L.ffsyrk_digit_planes.restype = i32
            L.ffsyrk_i8_schedule.argtypes = [u32, i32, P(i32), i32]
            L.ffsyrk_i8_schedule.restype = i32
            L.ffsyrk_i8_digit_bounds.argtypes = [u32, P(i32)]
            L.ffsyrk_i8_digit_bounds.restype = i32
            L.ffsyrk_digit_base.argtypes = [u32]
            L.ffsyrk_digit_base.restype = i32
            for name in ["ffsyrk_plan", "ffsyrk_plan_destroy", "ffsyrk_with_plan", "ffsyrk",
                         "ffsyrk_with_plan_update", "ffsyrk_update", "ffsyrkd_with_plan_update",
                         "ffsyrkd_update", "ffsyrkbd_with_plan_update", "ffsyrkbd_update",
                         "ffsyrk_noalloc",
                         "ffsyrk_batched", "ffsyrk_sync_status", "ffsyrk_plan_get_info",
                         "ffsyrk_plan_set_timing", "ffsyrk_plan_get_timing"]:
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def status_string(code: int) -> str:
    try:
        return lib().ffsyrk_status_string(code).decode()
    except FileNotFoundError:
        return f"status {code}"


def _check(code: int, where: str) -> None:
    if code != SUCCESS:
        raise FfsyrkError(code, where)


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _mat_args(X: torch.Tensor, name: str):
    if X.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if X.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise TypeError(f"{name} must hold uint32 bit patterns (torch.int32 or torch.uint32)")
    if X.numel() > 0 and X.stride(1) != 1:
        raise ValueError(f"{name} must have unit column stride")
    ld = max(X.stride(0), X.shape[1], 1) if X.shape[0] > 1 else max(X.shape[1], 1)
    return X.data_ptr(), ld


_PRODUCTS = {None: 0, "auto": 0, "schoolbook": 1, "karatsuba": 2}
_UNIT_BOUNDS = {None: 0, "data": 0, "worst": 1}


def make_options(leaf=None, levels=None, tile_ctas=None, autotune=False,
                 winograd=None, digit_products=None, epilogue_warps=0, unit_bounds=None) -> Options:
    """Plan options; winograd: None = automatic, 0 = off, w = at most w levels of Algorithm 1;
    digit_products: None/"auto", "schoolbook" or "karatsuba" (tensor-core leaf);
    unit_bounds: None/"data" (accumulator units from the operands' digits) or "worst"."""
    o = Options()
    lib().ffsyrk_options_default(ctypes.byref(o))
    o.leaf = _LEAVES[leaf] if not isinstance(leaf, int) else leaf
    o.levels = LEVELS_AUTO if levels is None else int(levels)
    o.tile_ctas = 0 if tile_ctas is None else int(tile_ctas)
    o.autotune = 1 if autotune else 0
    o.winograd = -1 if winograd is None else int(winograd)
    o.digit_products = _PRODUCTS[digit_products]
    o.epilogue_warps = int(epilogue_warps or 0)
    o.unit_bounds = _UNIT_BOUNDS[unit_bounds]
    return o


class Plan:
    """An ffsyrk plan: p, Y, digits, depth and workspace for n ≤ max_n, k ≤ max_k."""

    def __init__(self, p: int, max_n: int, max_k: int, leaf=None, levels=None, tile_ctas=None,
                 autotune=False, winograd=None, digit_products=None, epilogue_warps=0,
                 unit_bounds=None):
        self.p = int(p)
        self._h = ctypes.c_void_p()
        o = make_options(leaf, levels, tile_ctas, autotune, winograd, digit_products, epilogue_warps,
                         unit_bounds)
        _check(lib().ffsyrk_plan(ctypes.byref(self._h), self.p, int(max_n), int(max_k),
                                 ctypes.byref(o)), "ffsyrk_plan")

    def info(self) -> dict:
        i = PlanInfo()
        _check(lib().ffsyrk_plan_get_info(self._h, ctypes.byref(i)), "ffsyrk_plan_get_info")
        return {"p": i.p, "y_form": i.y_form, "y_a": i.y_a, "y_b": i.y_b, "y_cost": i.y_cost,
                "leaf": i.leaf, "levels": i.levels, "digits": i.digits,
                "chunk_k": list(i.chunk_k), "workspace_bytes": i.workspace_bytes,
                "tile_ctas": i.tile_ctas, "autotuned": i.autotuned, "tuned_ms": i.tuned_ms,
                "winograd": list(i.winograd), "planes": i.planes, "products": i.products,
                "epilogue_warps": i.epilogue_warps, "unit_bounds": i.unit_bounds}

    def __call__(self, A: torch.Tensor, C: torch.Tensor | None = None, uplo: str = "lower",
                 stream=None, alpha: int = 1, beta: int = 0) -> torch.Tensor:
        """C = A·Aᵀ mod p, or the update C ← α·A·Aᵀ + β·C mod p (triangle ``uplo``)."""
        n, k = A.shape
        if C is None:
            C = torch.zeros((n, n), dtype=torch.int32, device=A.device)
        pa, lda = _mat_args(A, "A")
        pc, ldc = _mat_args(C, "C")
        u = UPPER if uplo == "upper" else LOWER
        if (alpha, beta) == (1, 0):
            _check(lib().ffsyrk_with_plan(self._h, u, n, k, self.p, pa, lda, pc, ldc,
                                          _stream_handle(stream)), "ffsyrk_with_plan")
        else:
            _check(lib().ffsyrk_with_plan_update(self._h, u, n, k, self.p, int(alpha) & 0xFFFFFFFF,
                                                 pa, lda, int(beta) & 0xFFFFFFFF, pc, ldc,
                                                 _stream_handle(stream)), "ffsyrk_with_plan_update")
        return C

    def host(self, A: torch.Tensor, C: torch.Tensor, uplo: str = "lower", stream=None) -> torch.Tensor:
        """C = A·Aᵀ mod p for CPU tensors A (n × k) and C (n × n): copies A in, computes, and copies
        the n × n result back (the triangle ``uplo``, zeros in the other strict triangle), all
        enqueued on ``stream``; pin both tensors for asynchronous copies, and synchronise the
        stream before reading C."""
        if A.is_cuda or C.is_cuda:
            raise ValueError("host() takes CPU tensors")
        n, k = A.shape
        pa, lda = _mat_args(A, "A")
        pc, ldc = _mat_args(C, "C")
        _check(lib().ffsyrk_host(self._h, UPPER if uplo == "upper" else LOWER, n, k, self.p, pa,
                                 lda, pc, ldc, _stream_handle(stream)), "ffsyrk_host")
        return C

    def syrkd(self, A: torch.Tensor, d, C: torch.Tensor | None = None, uplo: str = "lower",
              stream=None, alpha: int = 1, beta: int = 0) -> torch.Tensor:
        """C ← α·A·Diag(d)·Aᵀ + β·C mod p (Algorithm 5); d holds k host values."""
        n, k = A.shape
        if C is None:
            C = torch.zeros((n, n), dtype=torch.int32, device=A.device)
        pa, lda = _mat_args(A, "A")
        pc, ldc = _mat_args(C, "C")
        dv = _u32_array(d, k)
        _check(lib().ffsyrkd_with_plan_update(self._h, UPPER if uplo == "upper" else LOWER, n, k,
                                              self.p, int(alpha) & 0xFFFFFFFF, pa, lda, dv,
                                              int(beta) & 0xFFFFFFFF, pc, ldc,
                                              _stream_handle(stream)), "ffsyrkd_with_plan_update")
        return C

    def syrkbd(self, A: torch.Tensor, d, e, C: torch.Tensor | None = None, uplo: str = "lower",
               stream=None, alpha: int = 1, beta: int = 0) -> torch.Tensor:
        """C ← α·A·B·Aᵀ + β·C mod p (Algorithm 6): B block diagonal, diagonal d, off-diagonal e."""
        n, k = A.shape
        if C is None:
            C = torch.zeros((n, n), dtype=torch.int32, device=A.device)
        pa, lda = _mat_args(A, "A")
        pc, ldc = _mat_args(C, "C")
        dv = _u32_array(d, k)
        ev = _u32_array(e, max(k - 1, 0)) if e is not None else None
        _check(lib().ffsyrkbd_with_plan_update(self._h, UPPER if uplo == "upper" else LOWER, n, k,
                                               self.p, int(alpha) & 0xFFFFFFFF, pa, lda, dv, ev,
                                               int(beta) & 0xFFFFFFFF, pc, ldc,
                                               _stream_handle(stream)), "ffsyrkbd_with_plan_update")
        return C

    def set_timing(self, enable: bool = True) -> None:
        _check(lib().ffsyrk_plan_set_timing(self._h, 1 if enable else 0), "ffsyrk_plan_set_timing")

    def timing(self) -> dict:
        t = Timing()
        _check(lib().ffsyrk_plan_get_timing(self._h, ctypes.byref(t)), "ffsyrk_plan_get_timing")
        return {f: getattr(t, f) for f, _ in Timing._fields_}

    def units(self, stream=None) -> tuple[int, int]:
        """(worst-case units, units the leaf ran) of the last tensor-core call (synchronises)."""
        h, u = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ffsyrk_plan_units(self._h, _stream_handle(stream), ctypes.byref(h),
                                       ctypes.byref(u)), "ffsyrk_plan_units")
        return h.value, u.value

    def selftest_timeout(self, limit_ns: int, stream=None) -> None:
        _check(lib().ffsyrk_plan_selftest_timeout(self._h, int(limit_ns), _stream_handle(stream)),
               "ffsyrk_plan_selftest_timeout")

    def sync_status(self, stream=None) -> None:
        _check(lib().ffsyrk_sync_status(self._h, _stream_handle(stream)), "ffsyrk_sync_status")

    def close(self) -> None:
        if self._h:
            lib().ffsyrk_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HerkPlan:
    """A plan for C = A·Aᴴ over F_{p²} = F_p[i]/(i² − r) (r a non-square mod p).

    A is an n × 2k int32/uint32 tensor of interleaved (Re, Im) residues; the
    result is the triangle ``uplo`` of Re C and Im C in two n × n tensors.
    """

    def __init__(self, p: int, r: int, max_n: int, max_k: int, leaf=None, levels=None,
                 tile_ctas=None, winograd=None):
        self.p, self.r = int(p), int(r)
        self._h = ctypes.c_void_p()
        o = make_options(leaf, levels, tile_ctas, False, winograd)
        _check(lib().ffherk_plan(ctypes.byref(self._h), self.p, self.r & 0xFFFFFFFF, int(max_n),
                                 int(max_k), ctypes.byref(o)), "ffherk_plan")

    def __call__(self, A: torch.Tensor, Cre: torch.Tensor | None = None,
                 Cim: torch.Tensor | None = None, uplo: str = "lower", stream=None):
        n, k2 = A.shape
        if k2 % 2:
            raise ValueError("A must hold (Re, Im) pairs: an even number of columns")
        if Cre is None:
            Cre = torch.zeros((n, n), dtype=torch.int32, device=A.device)
        if Cim is None:
            Cim = torch.zeros((n, n), dtype=torch.int32, device=A.device)
        pa, lda = _mat_args(A, "A")
        pr, ldr = _mat_args(Cre, "Cre")
        pi, ldi = _mat_args(Cim, "Cim")
        if ldr != ldi:
            raise ValueError("Cre and Cim must have the same row stride")
        _check(lib().ffherk_with_plan(self._h, UPPER if uplo == "upper" else LOWER, n, k2 // 2,
                                      pa, lda, pr, pi, ldr, _stream_handle(stream)),
               "ffherk_with_plan")
        return Cre, Cim

    def sync_status(self, stream=None) -> None:
        _check(lib().ffherk_sync_status(self._h, _stream_handle(stream)), "ffherk_sync_status")

    def close(self) -> None:
        if self._h:
            lib().ffherk_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def herk(A: torch.Tensor, p: int, r: int, uplo: str = "lower", Cre: torch.Tensor | None = None,
         Cim: torch.Tensor | None = None, stream=None):
    """(Re C, Im C) of C = A·Aᴴ over F_p[i]/(i² − r) through the plan cache (A interleaved)."""
    n, k2 = A.shape
    if k2 % 2:
        raise ValueError("A must hold (Re, Im) pairs: an even number of columns")
    if Cre is None:
        Cre = torch.zeros((n, n), dtype=torch.int32, device=A.device)
    if Cim is None:
        Cim = torch.zeros((n, n), dtype=torch.int32, device=A.device)
    pa, lda = _mat_args(A, "A")
    pr, ldr = _mat_args(Cre, "Cre")
    pi, ldi = _mat_args(Cim, "Cim")
    if ldr != ldi:
        raise ValueError("Cre and Cim must have the same row stride")
    _check(lib().ffherk(UPPER if uplo == "upper" else LOWER, n, k2 // 2, int(p),
                        int(r) & 0xFFFFFFFF, pa, lda, pr, pi, ldr, _stream_handle(stream)), "ffherk")
    return Cre, Cim


def workspace_query(p: int, max_n: int, max_k: int, leaf=None, levels=None, tile_ctas=None,
                    autotune=False, winograd=None, sms: int = 0,
                    digit_products=None) -> tuple[int, int]:
    """(workspace bytes, shared-tile slot bytes) a Plan with these arguments allocates (no GPU)."""
    o = make_options(leaf, levels, tile_ctas, autotune, winograd, digit_products)
    ws, sl = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().ffsyrk_workspace_query(int(p), int(max_n), int(max_k), ctypes.byref(o), int(sms),
                                        ctypes.byref(ws), ctypes.byref(sl)), "ffsyrk_workspace_query")
    return ws.value, sl.value


def leaf_schedule(p: int, kblocks: int) -> list[tuple[int, int, int, int, bool]]:
    """The leaf's K schedule for p: (i, j, first k-block, k-blocks, opens a unit)."""
    n = lib().ffsyrk_leaf_schedule(int(p), int(kblocks), None, 0)
    if n < 0:
        raise ValueError("bad p or kblocks")
    buf = (ctypes.c_int32 * (5 * max(n, 1)))()
    lib().ffsyrk_leaf_schedule(int(p), int(kblocks), buf, n)
    return [(buf[5 * q], buf[5 * q + 1], buf[5 * q + 2], buf[5 * q + 3], bool(buf[5 * q + 4]))
            for q in range(n)]


def leaf_schedule_ks(p: int, kblocks: int) -> list[tuple[int, int, int, int, bool]]:
    """The tensor-core leaf's K schedule with Karatsuba digit products: (i, i, first, count, opens a unit)."""
    n = lib().ffsyrk_leaf_schedule_ks(int(p), int(kblocks), None, 0)
    if n < 0:
        raise ValueError("bad p or kblocks")
    buf = (ctypes.c_int32 * (5 * max(n, 1)))()
    lib().ffsyrk_leaf_schedule_ks(int(p), int(kblocks), buf, n)
    return [(buf[5 * q], buf[5 * q + 1], buf[5 * q + 2], buf[5 * q + 3], bool(buf[5 * q + 4]))
            for q in range(n)]


def digit_planes(p: int) -> tuple[list[int], list[int]]:
    """Karatsuba digit planes of p: (bounds per plane, weight w_t per plane), or ([], []) if not used."""
    md, wt = (ctypes.c_int32 * 6)(), (ctypes.c_uint32 * 6)()
    n = lib().ffsyrk_digit_planes(int(p), md, wt)
    if n < 0:
        raise ValueError("bad p")
    return [md[t] for t in range(n)], [wt[t] for t in range(n)]


def i8_schedule(p: int, kblocks: int) -> list[tuple[int, int, int, int, bool]]:
    """The INT8 leaf's K schedule (128-wide k-blocks): (i, j, first k-block, k-blocks, opens a unit)."""
    n = lib().ffsyrk_i8_schedule(int(p), int(kblocks), None, 0)
    if n < 0:
        raise ValueError("bad p or kblocks")
    buf = (ctypes.c_int32 * (5 * max(n, 1)))()
    lib().ffsyrk_i8_schedule(int(p), int(kblocks), buf, n)
    return [(buf[5 * q], buf[5 * q + 1], buf[5 * q + 2], buf[5 * q + 3], bool(buf[5 * q + 4]))
            for q in range(n)]


def i8_digit_bounds(p: int) -> list[int]:
    """Bounds on the INT8 leaf's byte digits of residues mod p (255 below the signed top digit)."""
    out = (ctypes.c_int32 * 3)()
    D = lib().ffsyrk_i8_digit_bounds(int(p), out)
    if D < 0:
        raise ValueError("bad p")
    return [out[t] for t in range(D)]


def digit_bounds(p: int) -> list[int]:
    """Bounds on |digit t| of the signed digit split of residues mod p (base: digit_base)."""
    out = (ctypes.c_int32 * 3)()
    D = lib().ffsyrk_digit_bounds(int(p), out)
    if D < 0:
        raise ValueError("bad p")
    return [out[t] for t in range(D)]


def _u32_array(d, k: int):
    """k host values as a uint32 buffer for the library (wrapping like int(x) & 0xFFFFFFFF).

    A contiguous numpy uint32 array passes without a copy; anything else
    (lists, other integer dtypes, CPU tensors) is converted once by numpy.
    """
    if isinstance(d, torch.Tensor):
        d = d.detach().cpu().numpy()
    a = np.asarray(d)
    if a.dtype != np.uint32:
        if a.dtype == object or a.dtype.kind not in "iu":
            a = np.array([int(x) & 0xFFFFFFFF for x in a.reshape(-1)], dtype=np.uint64)
        a = (a.astype(np.int64, copy=False) & 0xFFFFFFFF) if a.dtype.kind == "i" else a
        a = a.astype(np.uint32)
    a = np.ascontiguousarray(a.reshape(-1))
    if a.shape[0] != k:
        raise ValueError("d must hold one entry per column of A (e: one fewer)")
    if k == 0:
        a = np.zeros(1, dtype=np.uint32)
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def syrkd(A: torch.Tensor, d, p: int, uplo: str = "lower", C: torch.Tensor | None = None,
          stream=None, alpha: int = 1, beta: int = 0) -> torch.Tensor:
    """C ← α·A·Diag(d)·Aᵀ + β·C mod p (Algorithm 5) through the plan cache."""
    n, k = A.shape
    if C is None:
        C = torch.zeros((n, n), dtype=torch.int32, device=A.device)
    pa, lda = _mat_args(A, "A")
    pc, ldc = _mat_args(C, "C")
    dv = _u32_array(d, k)
    _check(lib().ffsyrkd_update(UPPER if uplo == "upper" else LOWER, n, k, int(p),
                                int(alpha) & 0xFFFFFFFF, pa, lda, dv, int(beta) & 0xFFFFFFFF, pc, ldc,
                                _stream_handle(stream)), "ffsyrkd_update")
    return C


def syrkd_factor(p: int, d) -> tuple[int, list[int], list[int], list[int]]:
    """Algorithm 5's column transform for diagonal d: (columns of Ā, partner, u, v)."""
    k = len(d)
    dv = _u32_array(d, k)
    pt = (ctypes.c_int32 * (k + 1))()
    u = (ctypes.c_uint32 * (k + 1))()
    v = (ctypes.c_uint32 * (k + 1))()
    kk = lib().ffsyrkd_factor(int(p), k, dv, pt, u, v)
    if kk < 0:
        raise ValueError("bad p or d")
    return kk, list(pt[:kk]), list(u[:kk]), list(v[:kk])


def syrkbd(A: torch.Tensor, d, e, p: int, uplo: str = "lower", C: torch.Tensor | None = None,
           stream=None, alpha: int = 1, beta: int = 0) -> torch.Tensor:
    """C ← α·A·B·Aᵀ + β·C mod p (Algorithm 6) through the plan cache."""
    n, k = A.shape
    if C is None:
        C = torch.zeros((n, n), dtype=torch.int32, device=A.device)
    pa, lda = _mat_args(A, "A")
    pc, ldc = _mat_args(C, "C")
    dv = _u32_array(d, k)
    ev = _u32_array(e, max(k - 1, 0)) if e is not None else None
    _check(lib().ffsyrkbd_update(UPPER if uplo == "upper" else LOWER, n, k, int(p),
                                 int(alpha) & 0xFFFFFFFF, pa, lda, dv, ev, int(beta) & 0xFFFFFFFF,
                                 pc, ldc, _stream_handle(stream)), "ffsyrkbd_update")
    return C


def syrkbd_factor(p: int, d, e) -> tuple[int, list[list[tuple[int, int]]]]:
    """Algorithm 6's column mix for B (diagonal d, off-diagonal e): (columns of Ā, terms).

    terms[c] lists (source column of A, coefficient) with Ā_c = Σ coef·A_src.
    """
    k = len(d)
    dv = _u32_array(d, k)
    ev = _u32_array(e, max(k - 1, 0)) if e is not None else None
    src = (ctypes.c_int32 * (4 * (k + 1)))()
    w = (ctypes.c_uint32 * (4 * (k + 1)))()
    kk = lib().ffsyrkbd_factor(int(p), k, dv, ev, src, w)
    if kk < 0:
        raise ValueError("bad p, d or e (overlapping 2x2 blocks?)")
    return kk, [[(src[4 * c + t], w[4 * c + t]) for t in range(4) if src[4 * c + t] >= 0]
                for c in range(kk)]


def syrkbd_factor_device(p: int, d, e) -> tuple[int, list[list[tuple[int, int]]]]:
    """As :func:`syrkbd_factor`, computed by the device planner (needs a GPU)."""
    k = len(d)
    dv = _u32_array(d, k)
    ev = _u32_array(e, max(k - 1, 0)) if e is not None else None
    src = (ctypes.c_int32 * (4 * (k + 1)))()
    w = (ctypes.c_uint32 * (4 * (k + 1)))()
    kk = lib().ffsyrkbd_factor_device(int(p), k, dv, ev, src, w)
    if kk == -1:
        raise ValueError("bad p, d or e (overlapping 2x2 blocks?)")
    if kk < 0:
        raise FfsyrkError(ERR_CUDA, "ffsyrkbd_factor_device")
    return kk, [[(src[4 * c + t], w[4 * c + t]) for t in range(4) if src[4 * c + t] >= 0]
                for c in range(kk)]


def digit_base(p: int) -> int:
    """Base of the signed digit split of residues mod p (256, or balanced ≈ √p)."""
    b = lib().ffsyrk_digit_base(int(p))
    if b < 0:
        raise ValueError("bad p")
    return b


def syrk(A: torch.Tensor, p: int, uplo: str = "lower", C: torch.Tensor | None = None,
         stream=None, alpha: int = 1, beta: int = 0) -> torch.Tensor:
    """C = A·Aᵀ mod p, or C ← α·A·Aᵀ + β·C mod p (triangle ``uplo``), through the plan cache."""
    n, k = A.shape
    if C is None:
        C = torch.zeros((n, n), dtype=torch.int32, device=A.device)
    pa, lda = _mat_args(A, "A")
    pc, ldc = _mat_args(C, "C")
    u = UPPER if uplo == "upper" else LOWER
    if (alpha, beta) == (1, 0):
        _check(lib().ffsyrk(u, n, k, int(p), pa, lda, pc, ldc, _stream_handle(stream)), "ffsyrk")
    else:
        _check(lib().ffsyrk_update(u, n, k, int(p), int(alpha) & 0xFFFFFFFF, pa, lda,
                                   int(beta) & 0xFFFFFFFF, pc, ldc, _stream_handle(stream)),
               "ffsyrk_update")
    return C


def batched(As: list[torch.Tensor], p: int, Cs: list[torch.Tensor] | None = None,
            uplo: str = "lower", stream=None) -> list[torch.Tensor]:
    """C_t = A_t·A_tᵀ mod p for uneven problems, in one library call."""
    count = len(As)
    if Cs is None:
        Cs = [torch.zeros((a.shape[0], a.shape[0]), dtype=torch.int32, device=a.device) for a in As]
    I64 = ctypes.c_int64 * count
    VP = ctypes.c_void_p * count
    ns, ks, ldas, ldcs, pas, pcs = I64(), I64(), I64(), I64(), VP(), VP()
    for t, (a, c) in enumerate(zip(As, Cs)):
        ns[t], ks[t] = a.shape
        pas[t], ldas[t] = _mat_args(a, "A")
        pcs[t], ldcs[t] = _mat_args(c, "C")
    _check(lib().ffsyrk_batched(UPPER if uplo == "upper" else LOWER, count, ns, ks, int(p), pas,
                                ldas, pcs, ldcs, _stream_handle(stream)), "ffsyrk_batched")
    return Cs


def inject_alloc_failure(skip: int = 0, count: int = 1) -> int:
    """Test hook: after ``skip`` successful plan allocations, fail the next ``count``."""
    return int(lib().ffsyrk_test_inject_alloc_failure(int(skip), int(count)))


def cache_info() -> tuple[int, int]:
    """(plans the ffsyrk() cache holds on this device, release-and-retry events so far)."""
    plans, rel = ctypes.c_int32(), ctypes.c_int64()
    _check(lib().ffsyrk_cache_info(ctypes.byref(plans), ctypes.byref(rel)), "ffsyrk_cache_info")
    return plans.value, rel.value


PIPES = {"mma_s8s8": 0, "mma_u8s8": 1, "mma_u8u8": 2, "mad_wide_u32": 3, "mma_bf16": 4}


def probe_pipe(kind: str, iters: int = 4096, blocks: int = 0, reps: int = 5) -> float:
    """Measured multiply-adds per second of one arithmetic pipe (median of ``reps`` launches)."""
    dev = torch.cuda.current_device()
    if blocks <= 0:
        blocks = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    macs = ctypes.c_double()
    times = []
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _check(lib().ffsyrk_probe_pipe(PIPES[kind], int(iters), int(blocks), sink.data_ptr(),
                                       stream.cuda_stream, ctypes.byref(macs)), "ffsyrk_probe_pipe")
        e1.record(stream)
        torch.cuda.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    times.sort()
    return macs.value / (times[len(times) // 2] * 1e-3)
