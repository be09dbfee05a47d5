"""Pins for the CPU oracle: it is checked against facts other than itself.

Oracle A (CRS SpMV): dense brute force with exact integer data, row sums for
x = 1, identity / permutation / diagonal closed forms, and the exact rational
result within the a-priori rounding bound.
Oracle B (pJDS / ELLPACK-R conversion, Sect. 2.1): a hand-worked b = 4
fixture, structural invariants, round trip back to CRS, the special cases
b = 1 (plain JDS), one block (ELLPACK), constant row length, and the one-full-
row closed form (b+1)N - b.
Listings 1 and 2 run over oracle-B arrays must equal oracle A bit for bit (same
per-row order, same unfused operations).
Reduced-precision stores: binary32 against numpy, bfloat16 against hand-worked
ties, subnormals and overflow, and against torch's float32 -> bfloat16 cast for
float32-exact inputs.
"""
import json
import os

import numpy as np
import pytest

import synth
from synth import tiny
from tests import pins


def _int_x(n, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(-3, 4, size=n).astype(np.float64)


# ----------------------------------------------------------------------------- Oracle A

@pytest.mark.parametrize("seed", range(6))
def test_crs_spmv_equals_dense_bruteforce_exact(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    n_rows, n_cols = int(rng.integers(1, 65)), int(rng.integers(1, 65))
    A = tiny.random_lengths(n_rows, n_cols, max_len=n_cols, seed=seed, integer_values=True)
    x = _int_x(n_cols, seed + 100)
    y = oracle_lib.crs_spmv(A, x)
    assert pins.check_spmv_dense_exact(A, x, y) == []


@pytest.mark.parametrize("seed", range(4))
def test_crs_spmv_within_rounding_bound_of_exact(oracle_lib, seed):
    A = tiny.random_lengths(40, 50, max_len=50, seed=seed)
    x = np.random.default_rng(seed).uniform(-1, 1, 50)
    y = oracle_lib.crs_spmv(A, x)
    assert pins.check_spmv_error_bound(A, x, y) == []


def test_crs_spmv_row_sums(oracle_lib):
    A = tiny.random_lengths(300, 200, max_len=60, seed=3, integer_values=True)
    y = oracle_lib.crs_spmv(A, np.ones(200))
    sums = np.array([sum(A.val[A.row_ptr[i]:A.row_ptr[i + 1]].tolist()) for i in range(300)])
    assert np.array_equal(y, sums)


def test_crs_spmv_closed_forms(oracle_lib):
    n = 97
    x = np.random.default_rng(0).uniform(-1, 1, n)
    eye = tiny.from_dense(np.eye(n))
    assert np.array_equal(oracle_lib.crs_spmv(eye, x), x)
    sigma = np.random.default_rng(1).permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), sigma] = 1.0
    assert np.array_equal(oracle_lib.crs_spmv(tiny.from_dense(P), x), x[sigma])
    d = np.random.default_rng(2).uniform(0.5, 2.0, n)
    assert np.array_equal(oracle_lib.crs_spmv(tiny.from_dense(np.diag(d)), x), d * x)


def test_crs_spmv_empty_and_ragged(oracle_lib):
    A = tiny.from_lengths([0, 3, 0, 0, 5, 1, 0], 9, seed=5, integer_values=True)
    x = _int_x(9, 1)
    y = oracle_lib.crs_spmv(A, x)
    assert pins.check_spmv_dense_exact(A, x, y) == []
    assert y[0] == 0.0 and y[2] == 0.0 and y[6] == 0.0


def test_crs_absmv_and_rows(oracle_lib):
    A = tiny.random_lengths(50, 40, max_len=40, seed=9, integer_values=True)
    x = _int_x(40, 2)
    s = oracle_lib.crs_absmv(A, x)
    assert np.array_equal(s, np.abs(pins.dense_of(A)) @ np.abs(x))
    rows = np.array([0, 7, 49, 13], np.int64)
    ys, ss = oracle_lib.crs_spmv_rows(A, x, rows)
    assert np.array_equal(ys, (pins.dense_of(A) @ x)[rows])
    assert np.array_equal(ss, s[rows])


def test_crs_spmv_threads_do_not_change_result(oracle_lib):
    A = synth.banded_uniform(n=5000, hw=300, seed=11)
    x = synth.vector(A.n_cols, seed=11)
    oracle_lib.set_threads(1)
    y1 = oracle_lib.crs_spmv(A, x)
    oracle_lib.set_threads(max(2, os.cpu_count() or 2))
    y2 = oracle_lib.crs_spmv(A, x)
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("k", [1, 3, 8])
def test_crs_spmm_equals_dense_and_columnwise(oracle_lib, k):
    A = tiny.random_lengths(70, 40, max_len=40, seed=k, integer_values=True)
    X = np.random.default_rng(k).integers(-3, 4, (40, k)).astype(np.float64)
    Y = oracle_lib.crs_spmm(A, X)
    assert np.array_equal(Y, pins.dense_of(A) @ X)
    B = tiny.random_lengths(50, 60, max_len=30, seed=k + 10)
    Xf = np.random.default_rng(k + 1).uniform(-1, 1, (60, k))
    Yf = oracle_lib.crs_spmm(B, Xf)
    for c in range(k):  # same per-(row, column) order as the single product
        assert np.array_equal(Yf[:, c], oracle_lib.crs_spmv(B, Xf[:, c].copy()))
    # a transposed right-hand-side layout (column-major X) must be caught
    if k > 1:
        Xt = np.ascontiguousarray(Xf.T).reshape(Xf.shape)
        assert not np.array_equal(oracle_lib.crs_spmm(B, Xt), Yf)


# ----------------------------------------------------------------------------- Oracle B

def _golden(golden_dir):
    with open(os.path.join(golden_dir, "pjds_b4_example.json")) as fh:
        g = json.load(fh)
    dense = np.zeros((g["n_rows"], g["n_cols"]))
    for r, cols in enumerate(g["rows"]):
        for c in cols:
            dense[r, c] = 100 * r + c + 1
    return g, tiny.from_dense(dense)


def test_pjds_hand_worked_b4(oracle_lib, golden_dir):
    g, A = _golden(golden_dir)
    P = oracle_lib.pjds_convert(A, b=g["b"])
    for key in ("perm", "inv_perm", "row_len", "block_len", "col_start", "col"):
        assert np.array_equal(P[key], np.array(g[key])), key
    assert np.array_equal(P["val"], np.array(g["val"], np.float64))
    assert P["n_pad"] == g["n_pad"] and P["n_max"] == g["n_max"]
    y = oracle_lib.crs_spmv(A, np.array(g["x"], np.float64))
    assert np.array_equal(y, np.array(g["y"], np.float64))
    assert np.array_equal(oracle_lib.pjds_listing(P, np.array(g["x"], np.float64)), y)


def test_ellr_hand_worked(oracle_lib, golden_dir):
    g, A = _golden(golden_dir)
    E = oracle_lib.ellr_convert(A, pad_to=g["ellpack_pad_to"])
    assert E["n_stored"] == g["ellpack_n_stored"]
    assert np.array_equal(E["row_max"], np.array(g["ellpack_row_max"]))
    assert pins.check_ellr(A, E, g["ellpack_pad_to"]) == []


@pytest.mark.parametrize("b", [1, 4, 32, 64])
@pytest.mark.parametrize("seed", range(3))
def test_pjds_invariants_and_roundtrip(oracle_lib, b, seed):
    A = tiny.random_lengths(int(np.random.default_rng(seed).integers(1, 150)), 80, max_len=30, seed=seed)
    P = oracle_lib.pjds_convert(A, b=b)
    assert pins.check_pjds_structure(A, P, b) == []
    assert pins.check_pjds_roundtrip(A, P) == []


def test_pjds_permuted_columns_roundtrip(oracle_lib):
    A = tiny.random_lengths(90, 90, max_len=20, seed=4)
    P = oracle_lib.pjds_convert(A, b=32, permute_cols=True)
    assert pins.check_pjds_structure(A, P, 32) == []
    assert pins.check_pjds_roundtrip(A, P, permuted_cols=True) == []


def test_pjds_b1_is_plain_jds(oracle_lib):
    A = tiny.random_lengths(77, 60, max_len=25, seed=8)
    P = oracle_lib.pjds_convert(A, b=1)
    assert P["n_stored"] == A.nnz
    assert np.array_equal(P["block_len"], P["row_len"])
    assert np.all(P["col"] >= 0)


def test_pjds_single_block_is_ellpack(oracle_lib):
    A = tiny.random_lengths(50, 60, max_len=25, seed=12)
    P = oracle_lib.pjds_convert(A, b=64)
    E = oracle_lib.ellr_convert(A, pad_to=64)
    assert P["n_blocks"] == 1
    assert P["n_stored"] == 64 * P["n_max"] == E["n_stored"]


def test_constant_row_length_has_no_padding(oracle_lib):
    A = tiny.constant_length(96, 70, 9, seed=1)
    P = oracle_lib.pjds_convert(A, b=32)
    E = oracle_lib.ellr_convert(A, pad_to=32)
    assert P["n_stored"] == A.nnz == E["n_stored"]


@pytest.mark.parametrize("n,b", [(64, 32), (128, 32), (96, 4)])
def test_one_full_row_closed_form(oracle_lib, n, b):
    # Sect. 2.1: one full row, one entry elsewhere -> pJDS holds (b+1)N - b
    # nonzeros-plus-padding, plain ELLPACK holds N*N.
    A = tiny.one_full_row(n, full_row=n // 3)
    P = oracle_lib.pjds_convert(A, b=b)
    E = oracle_lib.ellr_convert(A, pad_to=b)
    assert P["n_stored"] == (b + 1) * n - b
    assert E["n_stored"] == n * n


@pytest.mark.parametrize("b", [32, 64])
def test_listings_equal_crs_bit_for_bit(oracle_lib, b):
    A = synth.banded_uniform(n=3000, hw=400, seed=21)
    x = synth.vector(A.n_cols, seed=21)
    y = oracle_lib.crs_spmv(A, x)
    P = oracle_lib.pjds_convert(A, b=b)
    assert np.array_equal(oracle_lib.pjds_listing(P, x), y)
    E = oracle_lib.ellr_convert(A, pad_to=32)
    assert np.array_equal(oracle_lib.ellr_listing(E, x), y)
    Pp = oracle_lib.pjds_convert(A, b=b, permute_cols=True)
    yp = oracle_lib.pjds_listing(Pp, x[Pp["perm"]], scatter=False)
    assert np.array_equal(yp, y[Pp["perm"]])


def test_empty_matrix_conversion(oracle_lib):
    A = tiny.from_lengths([0, 0, 0], 5)
    P = oracle_lib.pjds_convert(A, b=32)
    assert P["n_max"] == 0 and P["n_stored"] == 0 and P["n_pad"] == 32
    assert np.array_equal(P["col_start"], [0])
    assert np.array_equal(oracle_lib.crs_spmv(A, np.ones(5)), np.zeros(3))


# ----------------------------------------------------------------------------- reduced precision

def test_round_f32_matches_numpy(oracle_lib):
    v = np.random.default_rng(0).uniform(-1, 1, 10000) * np.exp2(np.random.default_rng(1).integers(-140, 120, 10000))
    assert np.array_equal(oracle_lib.round_f32(v), v.astype(np.float32).astype(np.float64))


def test_round_bf16_hand_worked():
    import oracle
    e = np.exp2
    cases = [
        (1.0, 1.0),
        (1 + e(-8), 1.0),                    # tie -> even (1.0)
        (1 + 3 * e(-8), 1 + e(-6)),          # tie -> even mantissa
        (1 + e(-8) + e(-30), 1 + e(-7)),     # just above the tie: rounding once, not via binary32
        (-(1 + e(-8) + e(-30)), -(1 + e(-7))),
        (e(-133), e(-133)),                  # smallest subnormal
        (e(-134), 0.0),                      # tie between 0 and 2^-133 -> 0
        (3 * e(-134), e(-132)),              # tie -> even
        (e(128) - e(120), e(128) - e(120)),  # largest finite
        (e(128) - e(119), np.inf),           # tie at the top -> inf
        (0.1, 0.10009765625),
    ]
    got = oracle.round_bf16(np.array([c[0] for c in cases]))
    for (v, want), g in zip(cases, got):
        assert g == want, (v, g, want)


def test_round_bf16_matches_torch_on_float32_inputs():
    torch = pytest.importorskip("torch")
    import oracle
    v = np.random.default_rng(5).standard_normal(20000).astype(np.float32)
    v *= np.exp2(np.random.default_rng(6).integers(-30, 30, 20000)).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_bf16(v.astype(np.float64)), want)


# ----------------------------------------------------------------------------- the pins catch planted mistakes

def test_pins_catch_planted_mistakes(oracle_lib):
    """Each pin must fail on an oracle output with a plausible mistake."""
    A = tiny.random_lengths(60, 50, max_len=20, seed=31, integer_values=True)
    x = _int_x(50, 7)
    y = oracle_lib.crs_spmv(A, x)
    assert pins.check_spmv_dense_exact(A, x, y) == []
    # dropped last term of every row
    y_drop = y.copy()
    for i in range(A.n_rows):
        k = A.row_ptr[i + 1] - 1
        if k >= A.row_ptr[i]:
            y_drop[i] -= A.val[k] * x[A.col[k]]
    assert pins.check_spmv_dense_exact(A, x, y_drop) != []
    # transposed operand: A^T applied to the leading part of x
    At = tiny.from_dense(pins.dense_of(A).T[:, :A.n_rows] if A.n_cols >= A.n_rows else pins.dense_of(A).T)
    if At.n_rows == A.n_rows and At.n_cols == len(x):
        assert pins.check_spmv_dense_exact(A, x, oracle_lib.crs_spmv(At, x)) != []
    # sign error
    assert pins.check_spmv_dense_exact(A, x, -y) != [] or np.all(y == 0)

    B = tiny.random_lengths(100, 40, max_len=15, seed=32)
    P = oracle_lib.pjds_convert(B, b=32)
    assert pins.check_pjds_structure(B, P, 32) == []
    # unstable tie-break
    Q = dict(P)
    lens = np.diff(B.row_ptr)[P["perm"]]
    k = int(np.nonzero(lens[:-1] == lens[1:])[0][0])
    perm = P["perm"].copy()
    perm[k], perm[k + 1] = perm[k + 1], perm[k]
    Q["perm"] = perm
    assert pins.check_pjds_structure(B, Q, 32) != []
    # ascending instead of descending sort
    Q = dict(P)
    Q["perm"] = P["perm"][::-1].copy()
    assert pins.check_pjds_structure(B, Q, 32) != []
    # padding to the global maximum instead of the block maximum
    Q = dict(P)
    Q["block_len"] = np.full_like(P["block_len"], P["n_max"])
    assert pins.check_pjds_structure(B, Q, 32) != []
    # an entry moved (off-by-one column offset)
    Q = dict(P)
    cs = P["col_start"].copy()
    cs[1] += 1
    Q["col_start"] = cs
    assert pins.check_pjds_structure(B, Q, 32) != []
    # a value in the wrong slot
    Q = dict(P)
    val = P["val"].copy()
    val[0], val[1] = val[1], val[0]
    Q["val"] = val
    assert pins.check_pjds_roundtrip(B, Q) != []
