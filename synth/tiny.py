"""Tiny hand-shaped CRS matrices for unit tests (numpy, seeded).

No arithmetic of the pJDS method lives here: these only build patterns (empty
rows, one full row, constant row length, ragged lengths) and values.
"""
from __future__ import annotations

import numpy as np

from . import Crs


def from_dense(d: np.ndarray) -> Crs:
    """CRS of the nonzero pattern of a dense array, columns ascending."""
    d = np.asarray(d, dtype=np.float64)
    n_rows, n_cols = d.shape
    rows, cols = np.nonzero(d)
    row_ptr = np.zeros(n_rows + 1, np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return Crs(n_rows, n_cols, row_ptr, cols.astype(np.int32), d[rows, cols].copy())


def from_lengths(lengths, n_cols: int, seed: int = 0, integer_values: bool = False) -> Crs:
    """Random matrix with prescribed row lengths (distinct random columns per
    row). integer_values draws values from {-4..-1, 1..4} so products and sums
    are exact in fp64."""
    rng = np.random.default_rng(seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    if np.any(lengths > n_cols) or np.any(lengths < 0):
        raise ValueError("row length outside [0, n_cols]")
    n_rows = len(lengths)
    row_ptr = np.zeros(n_rows + 1, np.int64)
    row_ptr[1:] = np.cumsum(lengths)
    col = np.empty(row_ptr[-1], np.int32)
    for i in range(n_rows):
        col[row_ptr[i]:row_ptr[i + 1]] = np.sort(rng.choice(n_cols, size=lengths[i], replace=False))
    if integer_values:
        mag = rng.integers(1, 5, size=row_ptr[-1])
        val = np.where(rng.random(row_ptr[-1]) < 0.5, -mag, mag).astype(np.float64)
    else:
        val = rng.uniform(-1.0, 1.0, size=row_ptr[-1])
    return Crs(n_rows, n_cols, row_ptr, col, val)


def random_lengths(n_rows: int, n_cols: int, max_len: int, seed: int = 0, p_empty: float = 0.1,
                   integer_values: bool = False) -> Crs:
    """Ragged random matrix: lengths uniform in [1, max_len], a fraction p_empty of empty rows."""
    rng = np.random.default_rng(seed + 7919)
    lengths = rng.integers(1, max_len + 1, size=n_rows)
    lengths[rng.random(n_rows) < p_empty] = 0
    return from_lengths(np.minimum(lengths, n_cols), n_cols, seed=seed, integer_values=integer_values)


def one_full_row(n: int, full_row: int = 0, seed: int = 0) -> Crs:
    """One fully populated row and a single entry (the diagonal) in every other
    row: the extreme case discussed for ELLPACK vs pJDS storage (Sect. 2.1)."""
    lengths = np.ones(n, np.int64)
    lengths[full_row] = n
    rng = np.random.default_rng(seed)
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum(lengths)
    col = np.empty(row_ptr[-1], np.int32)
    for i in range(n):
        col[row_ptr[i]:row_ptr[i + 1]] = np.arange(n) if i == full_row else [i]
    val = rng.uniform(-1.0, 1.0, size=row_ptr[-1])
    return Crs(n, n, row_ptr, col, val)


def constant_length(n_rows: int, n_cols: int, length: int, seed: int = 0) -> Crs:
    return from_lengths(np.full(n_rows, length), n_cols, seed=seed)
