"""Checks that pin the oracle to facts other than itself.

Each check returns a list of failure messages (empty = pass), so the same check
can be run on the oracle's output and, in the mutation tests, on outputs with a
planted mistake that the check must catch.

Facts used (Kreutzer et al., arXiv:1112.5588):
  - y = A x has a plain definition; with small integer data every fp64
    product and sum is exact, so it must equal a dense brute-force product.
  - pJDS (Sect. 2.1): rows sorted by descending length, blocks of b rows padded
    to their longest row, the padded matrix stored column by column, entry
    (i, j) of the sorted matrix at col_start[j] + i (Listing 2 addressing).
  - ELLPACK-R (Sect. 2.1, Listing 1): entry (i, j) at j*N_pad + i, rowmax[i]
    holds the row length.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def dense_of(A) -> np.ndarray:
    d = np.zeros((A.n_rows, A.n_cols), np.float64)
    for i in range(A.n_rows):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            d[i, A.col[k]] += A.val[k]
    return d


def exact_spmv(A, x) -> list:
    """Exact rational y = A x (brute force with Fractions)."""
    xs = [Fraction(float(v)) for v in x]
    out = []
    for i in range(A.n_rows):
        s = Fraction(0)
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            s += Fraction(float(A.val[k])) * xs[A.col[k]]
        out.append(s)
    return out


def check_spmv_dense_exact(A, x, y) -> list:
    """Integer data: y must equal the dense product exactly."""
    ref = dense_of(A) @ np.asarray(x, np.float64)
    bad = np.nonzero(ref != y)[0]
    return [f"row {i}: {y[i]} != dense {ref[i]}" for i in bad[:5]]


def check_spmv_error_bound(A, x, y) -> list:
    """Any evaluation order: |y_i - exact_i| <= gamma_n (|A||x|)_i with
    gamma_n = n u / (1 - n u), u = 2^-53, n = row length (Higham, Thm 3.5)."""
    ex = exact_spmv(A, x)
    fails = []
    u = 2.0 ** -53
    for i in range(A.n_rows):
        n = int(A.row_ptr[i + 1] - A.row_ptr[i])
        scale = sum(abs(float(A.val[k])) * abs(float(x[A.col[k]])) for k in range(A.row_ptr[i], A.row_ptr[i + 1]))
        g = n * u / (1 - n * u)
        err = abs(Fraction(float(y[i])) - ex[i])
        if err > Fraction(g * scale) * Fraction(1.0000001):
            fails.append(f"row {i}: error {float(err)} > bound {g * scale}")
    return fails


def check_pjds_structure(A, P: dict, b: int) -> list:
    """Invariants of a pJDS conversion that follow from Sect. 2.1 alone."""
    f = []
    n = A.n_rows
    lens = np.diff(A.row_ptr).astype(np.int64)
    perm, inv = np.asarray(P["perm"]), np.asarray(P["inv_perm"])
    n_pad = -(-n // b) * b
    if P["n_pad"] != n_pad:
        f.append(f"n_pad {P['n_pad']} != {n_pad}")
    if sorted(perm.tolist()) != list(range(n)):
        f.append("perm is not a bijection on 0..n-1")
        return f
    if not np.array_equal(inv[perm], np.arange(n)):
        f.append("inv_perm[perm[i]] != i")
    pl = lens[perm]
    if np.any(pl[:-1] < pl[1:]):
        f.append("rows not sorted by descending length")
    # stable: equal lengths keep ascending original index
    same = pl[:-1] == pl[1:]
    if np.any(perm[:-1][same] > perm[1:][same]):
        f.append("equal-length rows out of original order")
    rl = np.asarray(P["row_len"])
    if not np.array_equal(rl[:n], pl) or np.any(rl[n:] != 0):
        f.append("row_len != length of sorted row")
    bl = np.asarray(P["block_len"])
    want_bl = np.array([rl[k * b:(k + 1) * b].max(initial=0) for k in range(n_pad // b)], np.int64)
    if not np.array_equal(bl, want_bl):
        f.append("block_len != longest row of each block")
    if np.any(bl[:-1] < bl[1:]):
        f.append("block_len not non-increasing")
    cs = np.asarray(P["col_start"], np.int64)
    n_max = int(bl.max(initial=0))
    if P["n_max"] != n_max or len(cs) != n_max + 1 or cs[0] != 0:
        f.append("col_start has the wrong size or start")
        return f
    dlen = np.array([b * int(np.sum(bl > j)) for j in range(n_max)], np.int64)
    if not np.array_equal(np.diff(cs), dlen):
        f.append("col_start is not the prefix sum of the jagged-diagonal lengths")
    if cs[-1] != int(np.sum(b * bl)) or P["n_stored"] != cs[-1]:
        f.append("n_stored != sum_k b * block_len[k]")
    return f


def crs_from_pjds(P: dict, permuted_cols: bool = False):
    """Rebuild (row_ptr, col, val) of the original matrix from pJDS arrays via
    Listing 2 addressing col_start[j] + i; pads must be (col -1, val 0)."""
    n = P["n_rows"]
    perm, rl, cs = P["perm"], P["row_len"], P["col_start"]
    col, val = np.asarray(P["col"]), np.asarray(P["val"])
    rows = [None] * n
    pad_ok = True
    for i in range(P["n_pad"]):
        for j in range(P["n_max"]):
            o = cs[j] + i
            if o >= cs[j + 1]:
                continue
            if i < n and j < rl[i]:
                continue
            if col[o] != -1 or val[o] != 0.0:
                pad_ok = False
    for i in range(n):
        ent = []
        for j in range(rl[i]):
            o = cs[j] + i
            c = int(col[o])
            if permuted_cols:
                c = int(perm[c])
            ent.append((c, float(val[o])))
        rows[perm[i]] = ent
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    cols = np.array([c for r in rows for c, _ in r], np.int32)
    vals = np.array([v for r in rows for _, v in r], np.float64)
    return row_ptr, cols, vals, pad_ok


def check_pjds_roundtrip(A, P: dict, permuted_cols: bool = False) -> list:
    rp, c, v, pad_ok = crs_from_pjds(P, permuted_cols)
    f = []
    if not np.array_equal(rp, A.row_ptr):
        f.append("round trip: row_ptr differs")
    elif not np.array_equal(c, A.col):
        f.append("round trip: columns differ")
    elif not np.array_equal(v, A.val):
        f.append("round trip: values differ")
    if not pad_ok:
        f.append("pad entries are not (col -1, val 0)")
    return f


def check_ellr(A, E: dict, pad_to: int) -> list:
    f = []
    n = A.n_rows
    lens = np.diff(A.row_ptr)
    n_pad = -(-n // pad_to) * pad_to
    n_max = int(lens.max(initial=0))
    if E["n_pad"] != n_pad or E["n_max"] != n_max or E["n_stored"] != n_pad * n_max:
        f.append("ELLPACK-R sizes wrong")
        return f
    rm = np.asarray(E["row_max"])
    if not np.array_equal(rm[:n], lens) or np.any(rm[n:] != 0):
        f.append("rowmax != row length")
    col, val = np.asarray(E["col"]), np.asarray(E["val"])
    for i in range(n_pad):
        for j in range(n_max):
            o = j * n_pad + i
            if i < n and j < lens[i]:
                k = A.row_ptr[i] + j
                if col[o] != A.col[k] or val[o] != A.val[k]:
                    f.append(f"entry ({i},{j}) misplaced")
                    return f
            elif col[o] != -1 or val[o] != 0.0:
                f.append(f"pad ({i},{j}) not (-1, 0)")
                return f
    return f
