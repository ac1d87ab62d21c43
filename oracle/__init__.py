"""The oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct CPU statement of everything the GPU hot path
computes, written from the paper and from the definitions of the number
formats it uses.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import it.  It shares no code,
header, table or constant with the CUDA library, and it never imports the
library package.

Parts:

* :func:`gemm` / :func:`gemm_rows` — the FP64 triple-loop GEMM
  ``C = alpha*A*B + beta*C0`` (the matrix-multiply component of Sec. 2.1 /
  Table 2), in C (``gemm_ref.c``), OpenMP over rows.
* :mod:`oracle.numerics` — bf16 / e4m3 rounding and the per-tensor fp8 scale,
  the two-piece bf16 split, the relative Frobenius error.
* :mod:`oracle.mlp_ref` — the FP64 MLP cost model: forward, masked-MSE
  loss, backward, Adam.
* :mod:`oracle.selector_ref` — exhaustive (measure-every-variant) selection
  and the regret of a pick.
* :mod:`oracle.stencil_ref` — the thermal 2-D stencil (the hotspot-like
  second component): one explicit heat-equation step, array form and
  cell-by-cell form, float64.

Pinned by ``tests/test_oracle_*.py`` against closed forms, exact integer
arithmetic, exact rational brute force, library routines and finite
differences.  Parity unpinned: none of the functions above (the regret
*target* is an empirical metric and is not a function of the oracle).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i64 = ctypes.c_int64
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_gemm_f64.argtypes = [i64, i64, i64, ctypes.c_double, dp, i64,
                                        dp, i64, ctypes.c_double, dp, i64]
        lib.oracle_gemm_f64.restype = ctypes.c_int
        lib.oracle_gemm_rows_f64.argtypes = [
            i64, i64, i64, ctypes.c_double, dp, i64, dp, i64, ctypes.c_double,
            dp, i64, ctypes.POINTER(ctypes.c_int64), i64, dp]
        lib.oracle_gemm_rows_f64.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    """Host threads the C oracle's OpenMP loops use."""
    return int(_load().oracle_num_threads())


def gemm(A, B, alpha=1.0, beta=0.0, C0=None):
    """FP64 ``alpha*A@B + beta*C0`` by the plain triple loop.

    A is (M, K), B is (K, N); any real dtype, converted exactly to float64.
    C0 (M, N) is read only when beta != 0.  Returns a new float64 array.
    """
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    if beta != 0.0:
        if C0 is None:
            raise ValueError("beta != 0 needs C0")
        C = np.array(C0, dtype=np.float64, order="C", copy=True)
        if C.shape != (m, n):
            raise ValueError("C0 shape")
    else:
        C = np.zeros((m, n), dtype=np.float64)
    if m and n:
        rc = _load().oracle_gemm_f64(m, n, k, float(alpha), _dptr(A), k,
                                     _dptr(B), n, float(beta), _dptr(C), n)
        if rc != 0:
            raise RuntimeError("oracle_gemm_f64 failed")
    return C


def gemm_rows(A, B, rows, alpha=1.0, beta=0.0, C0=None):
    """Rows ``rows`` of ``alpha*A@B + beta*C0`` (FP64), shape (len(rows), N)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    out = np.zeros((len(rows), n), dtype=np.float64)
    if beta != 0.0:
        if C0 is None:
            raise ValueError("beta != 0 needs C0")
        C0 = np.ascontiguousarray(C0, dtype=np.float64)
        c0p = _dptr(C0)
    else:
        c0p = None
    if len(rows) and n:
        rc = _load().oracle_gemm_rows_f64(
            m, n, k, float(alpha), _dptr(A), k, _dptr(B), n, float(beta), c0p,
            n, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(rows),
            _dptr(out))
        if rc != 0:
            raise RuntimeError("oracle_gemm_rows_f64 failed")
    return out


def library_path() -> str:
    return _build.LIB


__all__ = ["gemm", "gemm_rows", "num_threads", "library_path"]
