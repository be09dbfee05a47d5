"""C-ABI library on the host (no GPU): it loads, exports every declared symbol,
and its CRS -> pJDS / ELLPACK-R conversion equals the oracle's bit for bit.
Error paths return statuses, never abort."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synth
from synth import tiny
from tests.conftest import ROOT


@pytest.fixture(scope="module")
def P():
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds
    return pjds


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = re.sub(r"#[^\n]*", "", src)
        for m in re.finditer(r"\b([A-Za-z_]\w*)\s*\(([^;{}()]*(?:\([^()]*\))?[^;{}()]*)\)\s*;", src):
            names.append(m.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol(P):
    names = _declared_functions()
    assert "pjds_spmv" in names and "ellr_create" in names and len(names) >= 12
    lib = ctypes.CDLL(P.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


@pytest.mark.parametrize("b", [32, 64])
def test_create_shape_equals_create(P, b):
    # the structure from the row lengths alone is pjds_create's, without col / val
    for A in (synth.hmep_like(n=20_000, seed=3), tiny.random_lengths(1037, 900, max_len=70, seed=5, p_empty=0.2),
              synth.zipf_rows(70_000, s=2.0, len_max=512, seed=2), tiny.from_lengths([0] * 40, 7)):
        for dt in ("f64", "bf16"):
            H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dt)
            S = P.pjds_create_shape(A.n_rows, A.n_cols, A.row_ptr, b=b, dtype=dt)
            for k in ("n_rows", "n_cols", "n_pad", "b", "n_blocks", "n_max", "nnz", "n_stored", "dtype", "n_plan"):
                assert getattr(S, k) == getattr(H, k), k
            for k in ("perm", "inv_perm", "block_len", "row_len", "col_start", "tile_order", "plan"):
                assert np.array_equal(getattr(S, k), getattr(H, k)), k
            assert len(S.col) == 0 and len(S.val) == 0
            assert S.pair_share == 0  # no columns to compare
            H.destroy()
            S.destroy()
    with pytest.raises(P.PjdsError):
        P.pjds_create_shape(3, 3, np.array([0, 2, 1, 4]), b=32)  # row_ptr decreases


def test_abi_version_and_struct_sizes(P):
    assert P.lib().pjds_version() == 6  # the binding itself checked the struct sizes on load


CASES = [
    ("banded", lambda: synth.banded_uniform(n=4000, hw=500, seed=3)),
    ("ragged", lambda: tiny.random_lengths(333, 120, max_len=60, seed=5, p_empty=0.2)),
    ("rect_wide", lambda: tiny.random_lengths(70, 500, max_len=90, seed=6)),
    ("rect_tall", lambda: tiny.random_lengths(900, 40, max_len=40, seed=7)),
    ("one_full_row", lambda: tiny.one_full_row(130, full_row=77)),
    ("zipf", lambda: synth.zipf_rows(5000, s=1.8, len_max=300, seed=8)),
    ("empty_rows_only", lambda: tiny.from_lengths([0] * 45, 10)),
    ("single_row", lambda: tiny.from_lengths([7], 9, seed=1)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("b", [32, 64, 256])
def test_pjds_create_matches_oracle_bit_exact(P, oracle_lib, name, make, b):
    A = make()
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b)
    R = oracle_lib.pjds_convert(A, b=b)
    for k in ("n_pad", "n_blocks", "n_max", "n_stored", "nnz"):
        assert getattr(H, k) == R[k], k
    for k in ("perm", "inv_perm", "block_len", "row_len", "col_start", "col"):
        assert np.array_equal(getattr(H, k), R[k]), k
    assert np.array_equal(H.val.view(np.uint64), R["val"].view(np.uint64))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_pjds_create_reduced_precision_values(P, oracle_lib, dtype):
    A = synth.hmep_like(n=20_000, seed=2)
    # exercise ties, subnormals and overflow in the bf16 path as well
    e = np.exp2
    special = np.array([1 + e(-8), 1 + 3 * e(-8), 1 + e(-8) + e(-30), e(-133), e(-134), 3 * e(-134),
                        e(128) - e(119), e(128) - e(120), -0.1, 1e-45, 3e38, -3.4e38])
    val = A.val.copy()
    val[:len(special)] = special
    A = A._replace(val=val)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, val, b=32, dtype=dtype)
    R = oracle_lib.pjds_convert(A, b=32)
    want = oracle_lib.round_f32(R["val"]) if dtype == "f32" else oracle_lib.round_bf16(R["val"])
    if dtype == "f32":
        got = H.val.astype(np.float64)
    else:
        got = (H.val.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.array_equal(got, want)
    assert np.array_equal(H.col, R["col"])


def test_pjds_create_permuted_columns(P, oracle_lib):
    A = synth.hmep_like(n=30_000, seed=4)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, permute_cols=True)
    R = oracle_lib.pjds_convert(A, b=32, permute_cols=True)
    assert np.array_equal(H.col, R["col"]) and np.array_equal(H.val, R["val"])


@pytest.mark.parametrize("name,make", CASES[:6], ids=[c[0] for c in CASES[:6]])
def test_ellr_create_matches_oracle_bit_exact(P, oracle_lib, name, make):
    A = make()
    H = P.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val)
    R = oracle_lib.ellr_convert(A, pad_to=32)
    for k in ("n_pad", "n_max", "n_stored"):
        assert getattr(H, k) == R[k], k
    assert np.array_equal(H.row_max, R["row_max"])
    assert np.array_equal(H.col, R["col"])
    assert np.array_equal(H.val, R["val"])


def test_storage_reduction_vs_ellpack(P):
    # Sect. 2.1: pJDS never stores more than ELLPACK, and far less for a wide
    # spread of row lengths.
    A = synth.zipf_rows(20_000, s=2.0, len_max=512, seed=1)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    E = P.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val)
    assert H.n_stored <= E.n_stored
    assert 1 - H.n_stored / E.n_stored > 0.9


def _status(P, fn, *args):
    with pytest.raises(P.PjdsError) as ei:
        fn(*args)
    return ei.value.code


def test_error_paths_return_status(P):
    A = tiny.random_lengths(40, 30, max_len=10, seed=2)
    EINVAL, EOVER = -1, -4
    assert _status(P, P.pjds_create, A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, 48) == EINVAL  # b % 32
    assert _status(P, P.pjds_create, A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, 0) == EINVAL
    bad_col = A.col.copy()
    bad_col[3] = A.n_cols
    assert _status(P, P.pjds_create, A.n_rows, A.n_cols, A.row_ptr, bad_col, A.val, 32) == EINVAL
    bad_rp = A.row_ptr.copy()
    bad_rp[5] = bad_rp[6] + 1
    assert _status(P, P.pjds_create, A.n_rows, A.n_cols, bad_rp, A.col, A.val, 32) == EINVAL
    bad_rp = A.row_ptr.copy()
    bad_rp[0] = 1
    assert _status(P, P.ellr_create, A.n_rows, A.n_cols, bad_rp, A.col, A.val) == EINVAL
    assert _status(P, P.pjds_create, A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, 32, 7) == EINVAL  # dtype
    assert _status(P, P.pjds_create, A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, 32, "f64", True) == EINVAL
    lib = P.lib()
    assert lib.pjds_create(1, 1, None, None, None, 32, 0, 0, None) == EINVAL
    assert lib.pjds_spmv(None, None, None, None) == EINVAL
    assert lib.ellr_spmv(None, None, None, None) == EINVAL
    assert lib.pjds_destroy(None) == 0
    assert b"NULL" in lib.pjds_last_error() or lib.pjds_last_error() == b""
    del EOVER


def test_spmv_argument_checks_without_gpu(P):
    # Invalid configurations and inconsistent matrix views are rejected on the
    # host; pjds_spmv_resolve runs the same checks as pjds_spmv_cfg but never
    # launches, so no fake pointer can reach a kernel.
    A = tiny.random_lengths(64, 64, max_len=8, seed=1)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    for bad in (dict(rows_per_thread=3), dict(rows_per_thread=2, threads_per_row=2),
                dict(block_threads=1000), dict(block_threads=48), dict(threads_per_row=1, unroll=3),
                dict(rows_per_thread=2, unroll=16), dict(rows_per_thread=4, unroll=8),
                dict(threads_per_row=2, unroll=8)):
        with pytest.raises(P.PjdsError) as ei:
            P.pjds_spmv_resolve(H, **bad)
        assert ei.value.code == -1, bad
    s = P._dev_struct_from_host(H)
    s.n_pad = 33
    out = P._LaunchS()
    assert P.lib().pjds_spmv_resolve(ctypes.byref(s), None, ctypes.byref(out)) == -1
    s = P._dev_struct_from_host(H)
    s.val = 8  # misaligned for 4-row vector loads
    cfg = P._LaunchS(4, 1, 256, 0)
    assert P.lib().pjds_spmv_resolve(ctypes.byref(s), ctypes.byref(cfg), ctypes.byref(out)) == -1
    assert P.lib().pjds_spmv(None, None, None, None) == -1


def test_gpu_test_configs_resolve_on_host(P):
    # every configuration the GPU tests launch is accepted by the library
    from tests.test_gpu_spmv import CONFIG_SHAPES, CONFIGS
    for _, make in CONFIG_SHAPES:
        A = make()
        H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
        for cfg in CONFIGS:
            r = P.pjds_spmv_resolve(H, **cfg)
            assert all(r[k] == v for k, v in cfg.items()), (cfg, r)
        assert P.pjds_spmv_resolve(H)["unroll"] in (4, 8)


def _band(n, length, long_row=-1, long_len=64):
    # n x n, row i holds columns i, i+1, ... (mod n); row long_row holds long_len
    lens = np.full(n, length, np.int64)
    if long_row >= 0:
        lens[long_row] = long_len
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum(lens)
    rows = np.repeat(np.arange(n), lens)
    col = ((rows + np.arange(row_ptr[-1]) - row_ptr[rows]) % n).astype(np.int32)
    return synth.Crs(n, n, row_ptr, col, np.ones(row_ptr[-1]))


ENTRY_BYTES = {"f64": 12, "f32": 8, "bf16": 6}


def _expected_threads_per_row(n_rows, n_max, nnz, dt):
    # the longest row's chain against the stream time of the product:
    # ratio = n_max * 2^20 / (nnz * entry bytes); T = 1 below 2, 2 below 8,
    # 4 below 64, else 8; then doubled while n_rows * T < 2^17 (integer form)
    num, den = n_max * 2**20, max(nnz, 1) * ENTRY_BYTES[dt]
    t = 1 if num < 2 * den else 2 if num < 8 * den else 4 if num < 64 * den else 8
    while t < 8 and n_rows * t < 2**17:
        t *= 2
    return t


def test_resolve_defaults(P):
    A = synth.hmep_like(n=10_000, seed=1)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    # 10k rows: one thread per row would leave the GPU short of threads
    assert P.pjds_spmv_resolve(H) == {"rows_per_thread": 1, "threads_per_row": 8, "block_threads": 128, "unroll": 4,
                                      "staged": 0, "index64": 0, "tile_order": -1, "plan": -1}
    # both sides of every threshold: the thread floor (2^17 rows at T = 1,
    # 2^16 at T = 2, ...) and the chain ratio (a long row of growing length)
    seen = set()
    cases = [(n, 3, -1, 0) for n in (600_000, 1 << 17, (1 << 17) - 1, 1 << 16, (1 << 16) - 1, 20_000)]
    cases += [(600_000, 3, 12345, L) for L in (41, 42, 164, 165, 1319, 1320, 5000)]
    cases += [(300_000, 4, 7, L) for L in (60, 200, 1400)]
    for n, length, long_row, long_len in cases:
        C = _band(n, length, long_row, long_len)
        n_max = int(np.diff(C.row_ptr).max())
        for dt in ("f64", "f32", "bf16"):
            HC = P.pjds_create(C.n_rows, C.n_cols, C.row_ptr, C.col, C.val, b=32, dtype=dt)
            r = P.pjds_spmv_resolve(HC)
            t = _expected_threads_per_row(n, n_max, C.nnz, dt)
            assert r["threads_per_row"] == t and r["rows_per_thread"] == 1, (n, long_len, dt, r, t)
            assert r["block_threads"] == (256 if t == 1 or dt == "f32" else 128), (n, dt, r)
            seen.add(t)
            HC.destroy()
    assert seen == {1, 2, 4, 8}
    Z = synth.zipf_rows(10_000, s=2.0, len_max=512, seed=1)
    HZ = P.pjds_create(Z.n_rows, Z.n_cols, Z.row_ptr, Z.col, Z.val, b=32)
    assert P.pjds_spmv_resolve(HZ)["threads_per_row"] == 8
    assert P.pjds_spmv_resolve(HZ, rows_per_thread=2)["threads_per_row"] == 1
    with pytest.raises(P.PjdsError):
        P.pjds_spmv_resolve(HZ, unroll=16)
    # the paper's matrix classes at full size keep one thread per row: a
    # block-dense (DLR-like) matrix of 280k rows of 144 entries
    D = synth.block_dense(70_000, 4, 36, 0.05, seed=2)
    for dt in ("f64", "f32", "bf16"):
        HD = P.pjds_create(D.n_rows, D.n_cols, D.row_ptr, D.col, D.val, b=32, dtype=dt)
        assert P.pjds_spmv_resolve(HD)["threads_per_row"] == 1, dt
        HD.destroy()


def test_resolve_large_matrix_defaults(P):
    # short rows, many of them: one thread per row on 256-thread CTAs, and two
    # rows per thread for fp32 / bf16 values from 2^21 rows on
    C = _band(1 << 21, 3)
    for dt, R in (("f64", 1), ("f32", 2), ("bf16", 2)):
        H = P.pjds_create(C.n_rows, C.n_cols, C.row_ptr, C.col, C.val, b=32, dtype=dt)
        r = P.pjds_spmv_resolve(H)
        assert (r["threads_per_row"], r["rows_per_thread"], r["block_threads"], r["unroll"]) == (1, R, 256, 4), (dt, r)
        # asking for several threads per row implies one row per thread
        assert P.pjds_spmv_resolve(H, threads_per_row=2)["rows_per_thread"] == 1
        s = P._dev_struct_from_host(H)
        s.val = 514  # not aligned for paired loads: one row per thread
        out = P._LaunchS()
        assert P.lib().pjds_spmv_resolve(ctypes.byref(s), None, ctypes.byref(out)) == 0
        assert out.rows_per_thread == 1
        H.destroy()
    C = _band((1 << 21) - 1, 3)
    H = P.pjds_create(C.n_rows, C.n_cols, C.row_ptr, C.col, C.val, b=32, dtype="f32")
    assert P.pjds_spmv_resolve(H)["rows_per_thread"] == 1


def test_resolve_tile_order_rule(P):
    # automatic: the traversal table from 2^20 rows on when the longest row is
    # at most 4 times the mean row length; 1 / -1 force it on / off
    big = P.pjds_create(*(lambda C: (C.n_rows, C.n_cols, C.row_ptr, C.col, C.val))(_band(1 << 20, 3)), b=32)
    assert P.pjds_spmv_resolve(big)["tile_order"] == 1
    assert P.pjds_spmv_resolve(big, threads_per_row=4)["tile_order"] == 1
    assert P.pjds_spmv_resolve(big, tile_order=-1)["tile_order"] == -1
    assert P.pjds_spmv_resolve(big, staged=1)["tile_order"] == -1
    small = P.pjds_create(*(lambda C: (C.n_rows, C.n_cols, C.row_ptr, C.col, C.val))(_band((1 << 20) - 1, 3)), b=32)
    assert P.pjds_spmv_resolve(small)["tile_order"] == -1
    assert P.pjds_spmv_resolve(small, tile_order=1)["tile_order"] == 1
    spread = P.pjds_create(*(lambda C: (C.n_rows, C.n_cols, C.row_ptr, C.col, C.val))(
        _band(1 << 20, 3, long_row=5)), b=32)  # longest 64 > 4 x mean (~3)
    assert P.pjds_spmv_resolve(spread)["tile_order"] == -1
    for bad in (2, -2):
        with pytest.raises(P.PjdsError):
            P.pjds_spmv_resolve(big, tile_order=bad)
    s = P._dev_struct_from_host(big)
    s.tile_order = None  # no table: forcing it is an error, automatic falls back
    cfg, out = P._LaunchS(0, 0, 0, 0, 0, 0, 1), P._LaunchS()
    assert P.lib().pjds_spmv_resolve(ctypes.byref(s), ctypes.byref(cfg), ctypes.byref(out)) == -1
    assert P.lib().pjds_spmv_resolve(ctypes.byref(s), None, ctypes.byref(out)) == 0 and out.tile_order == -1


def test_staged_option_resolves(P):
    A = synth.hmep_like(n=10_000, seed=1)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    r = P.pjds_spmv_resolve(H, staged=1)
    assert r["staged"] == 1 and r["rows_per_thread"] == 1 and r["threads_per_row"] == 1
    with pytest.raises(P.PjdsError):
        P.pjds_spmv_resolve(H, staged=1, rows_per_thread=2)
    s = P._dev_struct_from_host(H)
    s.val = 520  # 8-byte aligned only
    cfg = P._LaunchS(0, 0, 0, 0, 1)
    out = P._LaunchS()
    assert P.lib().pjds_spmv_resolve(ctypes.byref(s), ctypes.byref(cfg), ctypes.byref(out)) == -1


@pytest.mark.parametrize("b", [32, 64, 256])
def test_tile_order_definition(P, b):
    # the traversal table lists the 32-row tiles of the sorted matrix by the
    # original index of their first row (stable), tiles of padding rows last
    for A in (synth.hmep_like(n=20_000, seed=3), tiny.random_lengths(1037, 900, max_len=70, seed=5, p_empty=0.2),
              synth.zipf_rows(5_000, s=2.0, len_max=300, seed=2), tiny.from_lengths([0] * 40, 7)):
        H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b)
        n_t = H.n_pad // 32
        first = np.arange(n_t) * 32
        key = np.full(n_t, np.iinfo(np.int64).max)
        real = first < A.n_rows
        key[real] = H.perm[first[real]]
        want = np.argsort(key, kind="stable")
        assert np.array_equal(H.tile_order, want)
        assert np.array_equal(np.sort(H.tile_order), np.arange(n_t))
        # keys of consecutive tiles never decrease
        k = key[H.tile_order]
        assert np.all(k[1:] >= k[:-1])
        H.destroy()


def test_host_stream_argument_checks_without_gpu(P):
    # rejected on the host before any CUDA call (the device pointers are never used)
    A = tiny.random_lengths(64, 64, max_len=8, seed=1)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    s = P._dev_struct_from_host(H)
    lib, V, ref = P.lib(), ctypes.c_void_p, ctypes.byref
    xd, yd = (V * 2)(1024, 2048), (V * 2)(4096, 8192)
    xh, yh = (V * 1)(1 << 20), (V * 1)(1 << 21)
    assert lib.pjds_spmv_host_stream(ref(s), -1, xh, yh, xd, yd, None) == -1
    assert lib.pjds_spmv_host_stream(ref(s), 1, None, yh, xd, yd, None) == -1
    assert lib.pjds_spmv_host_stream(ref(s), 1, xh, yh, (V * 2)(1024, 1024), yd, None) == -1
    assert lib.pjds_spmv_host_stream(ref(s), 1, xh, yh, xd, (V * 2)(4096, 1024), None) == -1
    assert lib.pjds_spmv_host_stream(ref(s), 1, (V * 1)(None), yh, xd, yd, None) == -1
    assert lib.pjds_spmv_host_stream(ref(s), 1, xh, yh, (V * 2)(None, 2048), yd, None) == -1
    assert lib.pjds_spmv_host_stream(ref(s), 1, xh, yh, (V * 2)(8, 8), yd, None) == -1
    assert b"distinct" in lib.pjds_last_error()


def test_batch_lanes_checked_before_any_cuda_call(P):
    from paper_1112_5588_gb300 import batch as Bt
    A = tiny.random_lengths(64, 64, max_len=8, seed=1)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    s = (P._PjdsDevS * 1)(P._dev_struct_from_host(H))
    V, I = ctypes.c_void_p, ctypes.c_int32
    h = V()
    for bad in (3, 16, -1):
        rc = Bt._lib.pjds_batch_create_lanes(1, s, (V * 1)(4096), (V * 1)(8192), (I * 1)(bad), V(1 << 20), 1 << 20,
                                             ctypes.byref(h), None)
        assert rc == -1 and b"lanes" in P.lib().pjds_last_error()


def test_batch_rule_checked_before_any_cuda_call(P):
    from paper_1112_5588_gb300 import batch as Bt
    A = tiny.random_lengths(64, 64, max_len=8, seed=1)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32)
    s = (P._PjdsDevS * 1)(P._dev_struct_from_host(H))
    V, I = ctypes.c_void_p, ctypes.c_int32
    h = V()
    rc = Bt._lib.pjds_batch_create_rule(1, s, (V * 1)(4096), (V * 1)(8192), (I * 3)(4, 0, 64), V(1 << 20), 1 << 20,
                                        ctypes.byref(h), None)
    assert rc == -1 and b"min_len" in P.lib().pjds_last_error()
    us, best = (ctypes.c_double * 1)(), I()
    rc = Bt._lib.pjds_batch_tune_rule(1, s, (V * 1)(4096), (V * 1)(8192), (I * 3)(4, 16, 64), 1, 0, V(1 << 20),
                                      1 << 20, None, 0, us, ctypes.byref(best), None)
    assert rc == -1 and b"reps" in P.lib().pjds_last_error()


# ----------------------------------------------------------------------------- per-tile mapping (plan)

PLAN_CAP = {8: 32, 4: 64, 2: 128, 1: 256, 0: 512, 3: 1024}  # rows a tile of each kind maps


def _plan_kind(L):
    # 8 lanes from 256 entries, 4 from 64, 2 from 16; below: four rows per
    # thread for blocks of at most 2 entries, else two
    return 8 if L >= 256 else 4 if L >= 64 else 2 if L >= 16 else 3 if L <= 2 else 0


@pytest.mark.parametrize("make", [
    lambda: synth.zipf_rows(20_011, s=1.8, len_max=700, seed=5),
    lambda: tiny.random_lengths(1037, 900, max_len=300, seed=6, p_empty=0.3),
    lambda: synth.hmep_like(n=5_000, seed=7),
    lambda: tiny.constant_length(96, 70, 9, seed=1),
    lambda: tiny.from_lengths([0] * 70, 5),
    lambda: tiny.from_lengths([600] + [1] * 40 + [20] * 33, 700, seed=3),
])
@pytest.mark.parametrize("b", [32, 64])
def test_plan_definition(P, make, b):
    A = make()
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b)
    plan, bl = H.plan, H.block_len
    assert plan.shape == (H.n_plan, 4) and H.n_plan <= H.n_pad // 32
    if A.n_rows == 0:
        assert H.n_plan == 0
        return
    assert np.all(plan[:, 0] == 0) and np.all(plan[:, 2] > 0)
    # the tiles partition the sorted rows, start on multiples of 32 and hold
    # at most their kind's rows
    by_row = plan[np.argsort(plan[:, 1])]
    assert by_row[0, 1] == 0 and np.array_equal(by_row[1:, 1], by_row[:-1, 1] + by_row[:-1, 2])
    assert by_row[-1, 1] + by_row[-1, 2] == A.n_rows
    assert np.all(by_row[:, 1] % 32 == 0)
    for row0, rows, kind in by_row[:, 1:]:
        assert rows <= PLAN_CAP[int(kind)]
        kinds = {_plan_kind(int(bl[k])) for k in range(row0 // b, (row0 + rows - 1) // b + 1)}
        assert kinds == {int(kind)}, (row0, rows, kind, kinds)
    # a tile ends early only at the matrix's end or where the kind changes
    for (row0, rows, kind), nxt in zip(by_row[:, 1:], list(by_row[1:, 1:]) + [None]):
        if rows < PLAN_CAP[int(kind)] and nxt is not None:
            assert nxt[2] != kind or _plan_kind(int(bl[(row0 + rows) // b])) != kind
    # entries by work per lane, largest first (below 2^21 rows)
    costs = [_plan_cost(bl, b, *map(int, e[1:])) for e in plan]
    assert all(c0 >= c1 for c0, c1 in zip(costs, costs[1:]))


def _plan_cost(bl, b, row0, rows, kind):
    lanes = 1 if kind in (0, 3) else kind
    blocks = np.arange(row0, row0 + rows) // b
    return int(bl[blocks].astype(np.int64).sum()) // lanes


def test_plan_order_from_2_21_rows(P):
    # from 2^21 rows: the entries of several lanes per row first, by work per
    # lane, largest first; then the short-row entries (kinds 0 and 3) by the
    # original index of their first row
    Z = synth.zipf_rows(1 << 21, s=2.0, len_max=512, seed=5)
    H = P.pjds_create(Z.n_rows, Z.n_cols, Z.row_ptr, Z.col, Z.val, b=32)
    plan, bl = H.plan, H.block_len
    short = np.isin(plan[:, 3], (0, 3))
    n_long = int((~short).sum())
    assert 0 < n_long < len(plan)
    assert not short[:n_long].any() and short[n_long:].all()
    costs = [_plan_cost(bl, 32, *map(int, e[1:])) for e in plan[:n_long]]
    assert all(c0 >= c1 for c0, c1 in zip(costs, costs[1:]))
    first = H.perm[plan[n_long:, 1]]
    assert np.all(first[:-1] < first[1:])


def test_plan_resolve(P):
    Z = synth.zipf_rows(70_000, s=2.0, len_max=512, seed=8)     # longest row >> 4 x mean, >= 2^16 rows
    HZ = P.pjds_create(Z.n_rows, Z.n_cols, Z.row_ptr, Z.col, Z.val, b=32)
    # size thresholds: 2^16 rows (fp64), 2^17 (fp32), 2^18 (bf16)
    for n, want in ((65_535, (-1, -1, -1)), (65_536, (1, -1, -1)), (131_072, (1, 1, -1)), (262_144, (1, 1, 1))):
        Zn = synth.zipf_rows(n, s=2.0, len_max=512, seed=10)
        for dt, w in zip(("f64", "f32", "bf16"), want):
            Hn = P.pjds_create(Zn.n_rows, Zn.n_cols, Zn.row_ptr, Zn.col, Zn.val, b=32, dtype=dt)
            assert P.pjds_spmv_resolve(Hn)["plan"] == w, (n, dt)
            assert P.pjds_spmv_resolve(Hn, plan=1)["plan"] == 1
            Hn.destroy()
    M = synth.hmep_like(n=50_000, seed=9)                        # longest row < 4 x mean
    HM = P.pjds_create(M.n_rows, M.n_cols, M.row_ptr, M.col, M.val, b=32)
    assert P.pjds_spmv_resolve(HZ)["plan"] == 1
    assert P.pjds_spmv_resolve(HM)["plan"] == -1
    assert P.pjds_spmv_resolve(HM, plan=1)["plan"] == 1
    # asking for a uniform mapping switches the plan off
    for kw in (dict(threads_per_row=2), dict(rows_per_thread=2), dict(block_threads=128), dict(unroll=4),
               dict(staged=1), dict(tile_order=-1), dict(plan=-1)):
        assert P.pjds_spmv_resolve(HZ, **kw)["plan"] == -1, kw
    assert P.pjds_spmv_resolve(HZ, index64=1)["plan"] == 1
    for bad in (dict(plan=2), dict(plan=-2), dict(plan=1, staged=1)):
        with pytest.raises(P.PjdsError):
            P.pjds_spmv_resolve(HZ, **bad)
    # no plan, or arrays the vector loads cannot take: automatic falls back,
    # forcing is an error
    for field, value in (("plan", None), ("col", 516), ("val", 520), ("plan", 520)):
        s = P._dev_struct_from_host(HZ)
        setattr(s, field, value)
        out = P._LaunchS()
        assert P.lib().pjds_spmv_resolve(ctypes.byref(s), None, ctypes.byref(out)) == 0 and out.plan == -1, field
        cfg = P._LaunchS(0, 0, 0, 0, 0, 0, 0, 1)
        assert P.lib().pjds_spmv_resolve(ctypes.byref(s), ctypes.byref(cfg), ctypes.byref(out)) == -1, field
    s = P._dev_struct_from_host(HZ)
    s.n_plan = s.n_pad // 32 + 1
    assert P.lib().pjds_spmv_resolve(ctypes.byref(s), None, ctypes.byref(P._LaunchS())) == -1


def test_check_word_only_in_the_checked_build(P):
    # the normal build has no device-side extent checks: PJDS_EINVAL, no GPU call
    w = ctypes.c_uint64(123)
    assert P.lib().pjds_check_word(ctypes.byref(w), 0, None) == -1
    assert b"checked build" in P.lib().pjds_last_error()
    assert w.value == 123 or w.value == 0


def _pair_share(A, perm):
    """Per mille of entries equal to the paired sorted row's entry at the same
    position (rows perm[2k], perm[2k+1]), counted for both rows, rounded down."""
    lens = np.diff(A.row_ptr)
    matches = 0
    for k in range(A.n_rows // 2):
        a, c = perm[2 * k], perm[2 * k + 1]
        m = min(lens[a], lens[c])
        matches += int(np.sum(A.col[A.row_ptr[a]:A.row_ptr[a] + m] == A.col[A.row_ptr[c]:A.row_ptr[c] + m]))
    return (2000 * matches) // max(int(A.row_ptr[-1]), 1)


def test_pair_share(P):
    # hand-worked: rows of lengths 2, 2, 1, 1 (sorted order = original order);
    # rows 0 / 1 share column 0 at position 0, rows 2 / 3 share column 5:
    # 2 matches, counted for both rows, of 6 entries -> 666 per mille
    row_ptr = np.array([0, 2, 4, 5, 6], np.int64)
    col = np.array([0, 3, 0, 4, 5, 5], np.int32)
    H = P.pjds_create(4, 6, row_ptr, col, np.ones(6), b=32)
    assert H.pair_share == 666
    # an odd last row has no pair; an empty matrix has no entries
    H = P.pjds_create(3, 6, row_ptr[:4], col[:5], np.ones(5), b=32)
    assert H.pair_share == 2000 * 1 // 5
    assert P.pjds_create(5, 3, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0), b=32).pair_share == 0
    # block-structured rows share every column with their pair; the others barely
    for A, lo, hi in ((synth.block_dense(2_000, 4, 36, 0.05, seed=2), 1000, 1000),
                      (synth.block_dense(2_000, 2, 20, 0.05, seed=2), 1000, 1000),
                      (synth.hmep_like(n=40_000, seed=3), 0, 100),
                      (synth.banded_uniform(n=20_000, seed=3), 0, 100),
                      (synth.zipf_rows(30_000, s=2.0, len_max=300, seed=4), 0, 300)):
        for pc in (0, 1):
            if pc and A.n_rows != A.n_cols:
                continue
            H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, permute_cols=pc)
            want = _pair_share(A, H.perm)
            assert H.pair_share == want and lo <= want <= hi, (H.pair_share, want)


def test_resolve_pairs_rows_on_block_structured_matrices(P):
    # fp32 / bf16 take two rows per thread from 2^18 rows of >= 64 entries on
    # when paired rows share their columns; fp64, smaller matrices and
    # unshared long rows keep one row per thread
    D = synth.block_dense(70_000, 4, 36, 0.05, seed=2)  # 280k rows of 144, pair_share 1000
    for dt, R in (("f64", 1), ("f32", 2), ("bf16", 2)):
        H = P.pjds_create(D.n_rows, D.n_cols, D.row_ptr, D.col, D.val, b=32, dtype=dt)
        r = P.pjds_spmv_resolve(H)
        assert (r["threads_per_row"], r["rows_per_thread"], r["plan"]) == (1, R, -1), (dt, r)
        assert r["block_threads"] == (128 if R == 2 else 256), (dt, r)
        s = P._dev_struct_from_host(H)
        s.pair_share = 499
        out = P._LaunchS()
        assert P.lib().pjds_spmv_resolve(ctypes.byref(s), None, ctypes.byref(out)) == 0
        assert out.rows_per_thread == 1
        H.destroy()
    D2 = synth.block_dense(35_000, 4, 36, 0.05, seed=2)  # 140k rows
    H = P.pjds_create(D2.n_rows, D2.n_cols, D2.row_ptr, D2.col, D2.val, b=32, dtype="f32")
    assert P.pjds_spmv_resolve(H)["rows_per_thread"] == 1
    B = synth.banded_uniform(n=300_000, m_lo=60, m_hi=100, hw=2000, seed=3)  # long rows, nothing shared
    H = P.pjds_create(B.n_rows, B.n_cols, B.row_ptr, B.col, B.val, b=32, dtype="f32")
    assert H.pair_share < 100 and P.pjds_spmv_resolve(H)["rows_per_thread"] == 1
