"""CPU oracle for C = A·Aᵀ mod p (arXiv 2001.04109) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline / reference arm) may import this package.  It shares no code with
the CUDA library in ``paper_2001_04109_gb300``: it neither imports it nor is
imported by it.

Contents
--------
* ``syrk_oracle.c`` / :func:`syrk` / :func:`syrk_rows` -- the plain
  schoolbook definition of lower(A·Aᵀ) mod p in 64-bit integers (the result
  Algorithm 2 of the paper reaches exactly, Section 3).
* :func:`syrk_update` -- the definition of the update C ← α·A·Aᵀ + β·C mod
  p on one triangle (Section 4.2, Table 4), from :func:`syrk`.
* :func:`syrkd` -- the plain definition of A·D·Aᵀ mod p for a diagonal D
  (the product Algorithm 5, syrkd, computes; Section 5), in ``syrk_oracle.c``.
* :func:`syrkbd` -- the plain definition of A·B·Aᵀ mod p for a symmetric
  tridiagonal B, which holds Algorithm 6's block-diagonal B (Section 5).
* :func:`herk` -- the plain definition of A·Aᴴ over F_{p²} = F_p[i]/(i² − r)
  (Section 3.2, conjugate transposition), in ``syrk_oracle.c``.
* :mod:`oracle.field` -- primality, Legendre symbols, square roots and the
  skew-orthogonal Y of Section 3.1 (Prop. 3.2, Prop. 3.3, Algorithm 3).
* :mod:`oracle.alg2` -- Algorithm 2 itself written step by step over F_p in
  Python integers, for the block identities of the appendix proof; its
  general products optionally by :mod:`oracle.winograd` (Algorithm 1).
* :mod:`oracle.cost` -- the operation-count recurrences behind Table 5 and
  Eq. (complexity) of Theorem 4.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "syrk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``syrk_oracle.c`` with gcc into ``oracle/liboracle.so``."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u32, p = ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p
        lib.oracle_syrk_modp.argtypes = [i64, i64, u32, p, i64, p, i64, ctypes.c_int, ctypes.c_int]
        lib.oracle_syrk_modp.restype = ctypes.c_int
        lib.oracle_syrk_rows.argtypes = [i64, i64, u32, p, i64, p, i64, p, i64, ctypes.c_int]
        lib.oracle_syrk_rows.restype = ctypes.c_int
        lib.oracle_syrkd_modp.argtypes = [i64, i64, u32, p, i64, p, p, i64, ctypes.c_int, ctypes.c_int]
        lib.oracle_syrkd_modp.restype = ctypes.c_int
        lib.oracle_syrkbd_modp.argtypes = [i64, i64, u32, p, i64, p, p, p, i64, ctypes.c_int,
                                           ctypes.c_int]
        lib.oracle_syrkbd_modp.restype = ctypes.c_int
        lib.oracle_herk_modp.argtypes = [i64, i64, u32, u32, p, i64, p, p, i64, ctypes.c_int]
        lib.oracle_herk_modp.restype = ctypes.c_int
        _lib = lib
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _as_u32(A) -> np.ndarray:
    A = np.asarray(A)
    if A.dtype in (np.int32, np.uint32):
        A = A.view(np.uint32)
    elif A.dtype.kind in "iu":
        A = A.astype(np.uint64).astype(np.uint32)
    else:
        raise TypeError(f"integer matrix expected, got {A.dtype}")
    return np.ascontiguousarray(A)


def syrk(A, p: int, uplo: str = "lower", threads: int | None = None) -> np.ndarray:
    """Schoolbook A·Aᵀ mod p of an n×k matrix (entries any uint32).

    ``uplo`` is ``"lower"`` (j ≤ i written), ``"upper"`` (j ≥ i) or
    ``"full"`` (every entry computed on its own).  Unwritten entries are 0.
    Returns an n×n uint32 array.
    """
    A = _as_u32(A)
    if A.ndim != 2:
        raise ValueError("A must be 2-D")
    n, k = A.shape
    C = np.zeros((n, n), dtype=np.uint32)
    code = {"lower": 0, "upper": 1, "full": 2}[uplo]
    lib = _load()
    rc = lib.oracle_syrk_modp(n, k, p, A.ctypes.data, max(k, 1), C.ctypes.data, max(n, 1), code,
                              threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_syrk_modp rejected its arguments")
    return C


def syrk_update(A, p: int, alpha: int, C, beta: int, uplo: str = "lower",
                threads: int | None = None) -> np.ndarray:
    """C ← α·A·Aᵀ + β·C mod p on the triangle ``uplo`` (Section 4.2, Table 4).

    The definition entry by entry: (α·(A·Aᵀ)[i][j] + β·C[i][j]) mod p where
    the triangle is stored (j ≤ i for ``"lower"``, j ≥ i for ``"upper"``);
    every other entry of C is returned unchanged.  α, β are reduced mod p;
    C's triangle must hold residues < p.  Returns a new n×n uint32 array.
    """
    C = np.array(C, dtype=np.uint32, copy=True)
    n = C.shape[0]
    P = syrk(A, p, uplo, threads).astype(np.uint64)
    a, b = np.uint64(int(alpha) % p), np.uint64(int(beta) % p)
    mask = np.tril(np.ones((n, n), dtype=bool)) if uplo == "lower" else np.triu(np.ones((n, n), dtype=bool))
    upd = (a * P + b * C.astype(np.uint64)) % np.uint64(p)  # < 2·p² < 2^49
    C[mask] = upd[mask].astype(np.uint32)
    return C


def syrkd(A, d, p: int, uplo: str = "lower", threads: int | None = None) -> np.ndarray:
    """Schoolbook A·Diag(d)·Aᵀ mod p of an n×k matrix and k diagonal entries.

    Entries of A and d may be any uint32 (reduced mod p first).  ``uplo`` as
    for :func:`syrk`; unwritten entries are 0.  Returns an n×n uint32 array.
    """
    A = _as_u32(A)
    n, k = A.shape
    dv = np.ascontiguousarray(np.asarray(d, dtype=np.uint64).astype(np.uint32))
    if dv.shape != (k,):
        raise ValueError("d must hold one entry per column of A")
    C = np.zeros((n, n), dtype=np.uint32)
    code = {"lower": 0, "upper": 1, "full": 2}[uplo]
    rc = _load().oracle_syrkd_modp(n, k, p, A.ctypes.data, max(k, 1),
                                   dv.ctypes.data if k else None, C.ctypes.data, max(n, 1), code,
                                   threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_syrkd_modp rejected its arguments")
    return C


def syrkbd(A, d, e, p: int, uplo: str = "lower", threads: int | None = None) -> np.ndarray:
    """Schoolbook A·B·Aᵀ mod p, B symmetric tridiagonal: B[l][l] = d[l], B[l][l+1] = B[l+1][l] = e[l].

    Algorithm 6 (syrkbd) takes a block-diagonal B with 1×1 and 2×2 blocks,
    i.e. a tridiagonal B whose nonzero e[l] are never adjacent; the
    definition here holds for any symmetric tridiagonal B.  ``e`` has k − 1
    entries (or None).  Entries may be any uint32 (reduced mod p first).
    """
    A = _as_u32(A)
    n, k = A.shape
    dv = np.ascontiguousarray(np.asarray(d, dtype=np.uint64).astype(np.uint32))
    if dv.shape != (k,):
        raise ValueError("d must hold one entry per column of A")
    ev = None
    if e is not None and k > 1:
        ev = np.ascontiguousarray(np.asarray(e, dtype=np.uint64).astype(np.uint32))
        if ev.shape != (k - 1,):
            raise ValueError("e must hold k - 1 entries")
    C = np.zeros((n, n), dtype=np.uint32)
    code = {"lower": 0, "upper": 1, "full": 2}[uplo]
    rc = _load().oracle_syrkbd_modp(n, k, p, A.ctypes.data, max(k, 1),
                                    dv.ctypes.data if k else None,
                                    ev.ctypes.data if ev is not None else None, C.ctypes.data,
                                    max(n, 1), code, threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_syrkbd_modp rejected its arguments")
    return C


def herk(A, p: int, r: int, uplo: str = "lower") -> tuple[np.ndarray, np.ndarray]:
    """A·Aᴴ over F_{p²} = F_p[i]/(i² − r) by definition; A interleaved (n × 2k: Re, Im, ...).

    Returns (Re C, Im C) as n×n uint32 arrays, the triangle ``uplo`` written
    ("full": every entry, each computed on its own), the rest 0.
    """
    A = _as_u32(A)
    n, k2 = A.shape
    if k2 % 2:
        raise ValueError("A must hold (Re, Im) pairs: an even number of columns")
    Cre = np.zeros((n, n), dtype=np.uint32)
    Cim = np.zeros((n, n), dtype=np.uint32)
    code = {"lower": 0, "upper": 1, "full": 2}[uplo]
    rc = _load().oracle_herk_modp(n, k2 // 2, p, r, A.ctypes.data, max(k2, 1), Cre.ctypes.data,
                                  Cim.ctypes.data, max(n, 1), code)
    if rc != 0:
        raise ValueError("oracle_herk_modp rejected its arguments")
    return Cre, Cim


def syrk_rows(A, p: int, rows, threads: int | None = None) -> np.ndarray:
    """Full rows ``rows`` of A·Aᵀ mod p, as a len(rows)×n uint32 array."""
    A = _as_u32(A)
    n, k = A.shape
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(rows), n), dtype=np.uint32)
    lib = _load()
    rc = lib.oracle_syrk_rows(n, k, p, A.ctypes.data, max(k, 1), rows.ctypes.data, len(rows),
                              out.ctypes.data, max(n, 1), threads or default_threads())
    if rc != 0:
        raise ValueError("oracle_syrk_rows rejected its arguments")
    return out
