"""CPU oracle for pJDS / ELLPACK-R SpMV (fp64, plain loops) — test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. The library in ``paper_1112_5588_gb300`` never does,
and the two share no code. The arithmetic lives in ``oracle.c``, compiled with
``-ffp-contract=off`` (no fused multiply-add) into ``liboracle.so``.

Every function states the passage of Kreutzer et al., "Sparse matrix-vector
multiplication on GPGPU clusters" (arXiv:1112.5588) it follows; see oracle.c.
Pins for each function (dense brute force, closed forms, invariants, hand-worked
fixtures) are in tests/test_oracle_pins.py; the Krylov oracles (krylov.py) are
pinned in tests/test_oracle_krylov.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                           "-std=c11", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_set_threads.argtypes = [ci]
        lib.oracle_set_threads.restype = None
        lib.oracle_max_threads.restype = ci
        lib.oracle_crs_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.oracle_crs_spmv.restype = None
        lib.oracle_crs_absmv.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.oracle_crs_absmv.restype = None
        lib.oracle_crs_spmm.argtypes = [i64, vp, vp, vp, i64, vp, vp]
        lib.oracle_crs_spmm.restype = None
        lib.oracle_crs_spmv_rows.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp]
        lib.oracle_crs_spmv_rows.restype = None
        lib.oracle_pjds_shape.argtypes = [i64, vp, i64, vp]
        lib.oracle_pjds_shape.restype = ci
        lib.oracle_pjds_fill.argtypes = [i64, i64, vp, vp, vp, i64, ci, vp, vp, vp, vp, vp, vp, vp]
        lib.oracle_pjds_fill.restype = ci
        lib.oracle_ellr_shape.argtypes = [i64, vp, i64, vp]
        lib.oracle_ellr_shape.restype = ci
        lib.oracle_ellr_fill.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp]
        lib.oracle_ellr_fill.restype = ci
        lib.oracle_pjds_listing.argtypes = [i64, vp, vp, vp, vp, vp, vp, ci, vp]
        lib.oracle_pjds_listing.restype = None
        lib.oracle_ellr_listing.argtypes = [i64, i64, vp, vp, vp, vp, vp]
        lib.oracle_ellr_listing.restype = None
        lib.oracle_round_f32.argtypes = [vp, vp, i64]
        lib.oracle_round_f32.restype = None
        lib.oracle_round_bf16.argtypes = [vp, vp, i64]
        lib.oracle_round_bf16.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def crs_spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x, fp64, CRS order, no fused multiply-add."""
    rp, col, val, x = _c(A.row_ptr, np.int64), _c(A.col, np.int32), _c(A.val, np.float64), _c(x, np.float64)
    y = np.empty(A.n_rows, np.float64)
    _load().oracle_crs_spmv(A.n_rows, _p(rp), _p(col), _p(val), _p(x), _p(y))
    return y


def crs_absmv(A, x: np.ndarray) -> np.ndarray:
    """|A| |x| (row-wise scale of the forward error bound)."""
    rp, col, val, x = _c(A.row_ptr, np.int64), _c(A.col, np.int32), _c(A.val, np.float64), _c(x, np.float64)
    s = np.empty(A.n_rows, np.float64)
    _load().oracle_crs_absmv(A.n_rows, _p(rp), _p(col), _p(val), _p(x), _p(s))
    return s


def crs_spmm(A, X: np.ndarray) -> np.ndarray:
    """Y = A X, X of shape (n_cols, k), fp64, CRS order for every column."""
    X = _c(X, np.float64)
    k = X.shape[1]
    rp, col, val = _c(A.row_ptr, np.int64), _c(A.col, np.int32), _c(A.val, np.float64)
    Y = np.empty((A.n_rows, k), np.float64)
    _load().oracle_crs_spmm(A.n_rows, _p(rp), _p(col), _p(val), k, _p(X), _p(Y))
    return Y


def crs_spmv_rows(A, x: np.ndarray, rows: np.ndarray):
    """(y[rows], (|A||x|)[rows]) for selected rows, for sampled checks at full size."""
    rp, col, val, x = _c(A.row_ptr, np.int64), _c(A.col, np.int32), _c(A.val, np.float64), _c(x, np.float64)
    rows = _c(rows, np.int64)
    y = np.empty(len(rows), np.float64)
    s = np.empty(len(rows), np.float64)
    _load().oracle_crs_spmv_rows(_p(rp), _p(col), _p(val), _p(x), _p(rows), len(rows), _p(y), _p(s))
    return y, s


def pjds_convert(A, b: int = 32, permute_cols: bool = False) -> dict:
    """pJDS arrays of A (Sect. 2.1) as a dict of numpy arrays plus sizes."""
    lib = _load()
    rp = _c(A.row_ptr, np.int64)
    sh = np.zeros(4, np.int64)
    if lib.oracle_pjds_shape(A.n_rows, _p(rp), b, _p(sh)):
        raise ValueError("oracle_pjds_shape failed")
    n_pad, n_blocks, n_max, n_stored = (int(v) for v in sh)
    out = dict(n_rows=A.n_rows, n_cols=A.n_cols, b=b, n_pad=n_pad, n_blocks=n_blocks, n_max=n_max,
               n_stored=n_stored, nnz=A.nnz,
               perm=np.empty(A.n_rows, np.int32), inv_perm=np.empty(A.n_rows, np.int32),
               block_len=np.empty(n_blocks, np.int32), row_len=np.empty(n_pad, np.int32),
               col_start=np.empty(n_max + 1, np.int64), col=np.empty(n_stored, np.int32),
               val=np.empty(n_stored, np.float64))
    col, val = _c(A.col, np.int32), _c(A.val, np.float64)
    rc = lib.oracle_pjds_fill(A.n_rows, A.n_cols, _p(rp), _p(col), _p(val), b, 1 if permute_cols else 0,
                              _p(out["perm"]), _p(out["inv_perm"]), _p(out["block_len"]), _p(out["row_len"]),
                              _p(out["col_start"]), _p(out["col"]), _p(out["val"]))
    if rc:
        raise ValueError("oracle_pjds_fill failed")
    return out


def ellr_convert(A, pad_to: int = 32) -> dict:
    """ELLPACK-R arrays of A (Sect. 2.1): element (i, j) at j*n_pad + i."""
    lib = _load()
    rp = _c(A.row_ptr, np.int64)
    sh = np.zeros(3, np.int64)
    if lib.oracle_ellr_shape(A.n_rows, _p(rp), pad_to, _p(sh)):
        raise ValueError("oracle_ellr_shape failed")
    n_pad, n_max, n_stored = (int(v) for v in sh)
    out = dict(n_rows=A.n_rows, n_cols=A.n_cols, n_pad=n_pad, n_max=n_max, n_stored=n_stored, nnz=A.nnz,
               row_max=np.empty(n_pad, np.int32), col=np.empty(n_stored, np.int32),
               val=np.empty(n_stored, np.float64))
    col, val = _c(A.col, np.int32), _c(A.val, np.float64)
    if lib.oracle_ellr_fill(A.n_rows, _p(rp), _p(col), _p(val), pad_to, _p(out["row_max"]), _p(out["col"]),
                            _p(out["val"])):
        raise ValueError("oracle_ellr_fill failed")
    return out


def pjds_listing(P: dict, x: np.ndarray, scatter: bool = True) -> np.ndarray:
    """Listing 2's loop, sequential, over converted pJDS arrays."""
    x = _c(x, np.float64)
    n_out = P["n_rows"]
    y = np.zeros(n_out, np.float64)
    _load().oracle_pjds_listing(P["n_rows"], _p(P["perm"]), _p(P["row_len"]), _p(P["col_start"]),
                                _p(P["col"]), _p(_c(P["val"], np.float64)), _p(x), 1 if scatter else 0, _p(y))
    return y


def ellr_listing(E: dict, x: np.ndarray) -> np.ndarray:
    """Listing 1's loop, sequential, over converted ELLPACK-R arrays."""
    x = _c(x, np.float64)
    y = np.zeros(E["n_rows"], np.float64)
    _load().oracle_ellr_listing(E["n_rows"], E["n_pad"], _p(E["row_max"]), _p(E["col"]),
                                _p(_c(E["val"], np.float64)), _p(x), _p(y))
    return y


def round_f32(v: np.ndarray) -> np.ndarray:
    v = _c(v, np.float64)
    out = np.empty_like(v)
    _load().oracle_round_f32(_p(v), _p(out), len(v))
    return out


def round_bf16(v: np.ndarray) -> np.ndarray:
    v = _c(v, np.float64)
    out = np.empty_like(v)
    _load().oracle_round_bf16(_p(v), _p(out), len(v))
    return out
