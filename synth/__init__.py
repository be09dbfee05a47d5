"""Seeded synthetic sparse matrices (CRS) shaped like the paper's test matrices.

This module is shared by the CUDA path's tests and bench and by the CPU oracle.
It holds no arithmetic of the pJDS method: it only draws matrices and vectors.
The heavy generators live in ``synth.c`` (built into ``libsynth.so`` by
``build()``); the tiny hand-shaped cases used by unit tests live in ``tiny.py``.

A CRS matrix is returned as a ``Crs`` named tuple of numpy arrays:
``row_ptr`` (int64, n_rows+1), ``col`` (int32, nnz, ascending within a row),
``val`` (float64, nnz), plus ``n_rows``, ``n_cols`` and ``param`` (a recorded
generator parameter, e.g. the geometric p of the HMEp-like matrix).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")


class Crs(NamedTuple):
    n_rows: int
    n_cols: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    param: float = 0.0

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def build(force: bool = False) -> str:
    """Compile libsynth.so with gcc (OpenMP, -fPIC); skipped when up to date."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32, f64, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
        lib.synth_banded_uniform.restype = vp
        lib.synth_banded_uniform.argtypes = [i64, i32, i32, i64, u64]
        lib.synth_hmep.restype = vp
        lib.synth_hmep.argtypes = [i64, i32, i32, i32, i32, i32, f64, u64]
        lib.synth_stencil27.restype = vp
        lib.synth_stencil27.argtypes = [i64, f64, u64]
        lib.synth_block_dense.restype = vp
        lib.synth_block_dense.argtypes = [i64, i32, i32, f64, u64]
        lib.synth_zipf.restype = vp
        lib.synth_zipf.argtypes = [i64, f64, i32, i32, i64, u64]
        for name in ("synth_nnz", "synth_n_rows", "synth_n_cols"):
            getattr(lib, name).restype = i64
            getattr(lib, name).argtypes = [vp]
        lib.synth_param.restype = f64
        lib.synth_param.argtypes = [vp]
        lib.synth_take.restype = None
        lib.synth_take.argtypes = [vp, vp, vp, vp]
        lib.synth_vector.restype = None
        lib.synth_vector.argtypes = [vp, i64, u64, u64]
        lib.synth_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _take(h) -> Crs:
    lib = _load()
    if not h:
        raise ValueError("synthetic generator rejected its parameters")
    n_rows, n_cols, nnz = lib.synth_n_rows(h), lib.synth_n_cols(h), lib.synth_nnz(h)
    param = lib.synth_param(h)
    row_ptr = np.empty(n_rows + 1, np.int64)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    lib.synth_take(h, row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    return Crs(int(n_rows), int(n_cols), row_ptr, col, val, float(param))


def banded_uniform(n: int = 20_000, m_lo: int = 5, m_hi: int = 40, hw: int = 2_000, seed: int = 1234) -> Crs:
    """Square n x n: row i = diagonal + (m_i-1) distinct columns uniform in
    [i-hw, i+hw], m_i uniform in [m_lo, m_hi]. Default: the small banded case
    (N = 20,000, ~450k nonzeros)."""
    return _take(_load().synth_banded_uniform(n, m_lo, m_hi, hw, seed))


def hmep_like(n: int = 6_200_000, offsets=(1, 64, 4096), m_lo: int = 2, m_hi: int = 14,
              target_nzr: float = 15.0, seed: int = 1234) -> Crs:
    """Holstein-Hubbard-like (HMEp, Sect. 1.3): 7 fixed diagonals plus symmetric
    random off-band entries within |j-i| <= n/8, ~target_nzr nonzeros per row."""
    o1, o2, o3 = offsets
    return _take(_load().synth_hmep(n, o1, o2, o3, m_lo, m_hi, target_nzr, seed))


def stencil27(g: int = 165, p_drop: float = 0.1, seed: int = 1234) -> Crs:
    """FEM-like SPD matrix: 27-point stencil on a g^3 grid, off-diagonal pairs
    dropped with probability p_drop, diagonal = sum|offdiag| + 1."""
    return _take(_load().synth_stencil27(g, p_drop, seed))


def block_dense(n_brow: int = 70_000, bs: int = 4, nb: int = 36, frac: float = 0.05, seed: int = 1234) -> Crs:
    """DLR-like (Sect. 1.3): dense bs x bs blocks, nb block columns per block
    row within ±frac of the block dimension; N = n_brow*bs, nb*bs per row."""
    return _take(_load().synth_block_dense(n_brow, bs, nb, frac, seed))


def zipf_rows(n: int, s: float = 2.0, len_max: int = 512, banded: bool = False, bw: int = 0,
              seed: int = 1234) -> Crs:
    """Power-law row lengths (Zipf exponent s, capped at len_max), distinct
    columns uniform over [0, n) or within ±bw of the row."""
    return _take(_load().synth_zipf(n, s, len_max, 1 if banded else 0, bw, seed))


def vector(n: int, seed: int = 1234, stream: int = 0) -> np.ndarray:
    """Dense float64 vector, entries uniform in [-1, 1)."""
    x = np.empty(n, np.float64)
    if n:
        _load().synth_vector(x.ctypes.data, n, seed, stream)
    return x


def threads() -> int:
    return int(_load().synth_threads())
