"""GPU parity: pjds_spmv / ellr_spmv through the C ABI against the CPU oracle.

Each case compares every output element with the oracle's y = A x on the same
seeded input, within the tolerances in tests/parity.py.
"""
import numpy as np
import pytest

import synth
from synth import tiny
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds
    return pjds


def _torch():
    import torch
    return torch


def run_pjds(P, A, x, b=32, dtype="f64", permute_cols=False, cfg=None):
    torch = _torch()
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dtype, permute_cols=permute_cols)
    D = H.to_device("cuda")
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=D.vec_dtype)
    y = torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
    if cfg is None:
        P.pjds_spmv(D, xt, y)
    else:
        P.pjds_spmv_cfg(D, xt, y, **cfg)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64), H, D


def run_ellr(P, A, x, dtype="f64"):
    torch = _torch()
    H = P.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype=dtype)
    D = H.to_device("cuda")
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=D.vec_dtype)
    y = torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
    P.ellr_spmv(D, xt, y)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def oracle_ref(oracle_lib, A, x):
    return oracle_lib.crs_spmv(A, x), oracle_lib.crs_absmv(A, x), np.diff(A.row_ptr)


SHAPES = [
    ("banded_20k", lambda: synth.banded_uniform(n=20_000, seed=1234)),
    ("ragged_tail", lambda: tiny.random_lengths(1037, 800, max_len=70, seed=3, p_empty=0.15)),
    ("rect_wide", lambda: tiny.random_lengths(301, 5000, max_len=200, seed=4)),
    ("rect_tall", lambda: tiny.random_lengths(4097, 33, max_len=33, seed=5)),
    ("one_full_row", lambda: tiny.one_full_row(700, full_row=500)),
    ("hmep_small", lambda: synth.hmep_like(n=100_000, seed=7)),
    ("zipf", lambda: synth.zipf_rows(60_000, s=2.0, len_max=512, seed=8)),
    ("single", lambda: tiny.from_lengths([3], 5, seed=2)),
]


CONFIGS = [
    dict(rows_per_thread=1, block_threads=128), dict(rows_per_thread=1, block_threads=512),
    dict(rows_per_thread=2), dict(rows_per_thread=4), dict(rows_per_thread=4, block_threads=64),
    dict(threads_per_row=2), dict(threads_per_row=4), dict(threads_per_row=8, block_threads=512),
    dict(threads_per_row=1, unroll=4), dict(threads_per_row=1, unroll=16), dict(rows_per_thread=2, unroll=8), dict(rows_per_thread=2, unroll=2),
    dict(rows_per_thread=4, unroll=4), dict(threads_per_row=4, unroll=2), dict(threads_per_row=2, block_threads=32),
    dict(staged=1), dict(index64=1), dict(threads_per_row=4, index64=1), dict(rows_per_thread=2, index64=1),
    dict(plan=1), dict(plan=1, index64=1),
]
CONFIG_SHAPES = [SHAPES[1], SHAPES[4], SHAPES[6]]


@pytest.mark.parametrize("name,make", SHAPES, ids=[s[0] for s in SHAPES])
@pytest.mark.parametrize("b", [32, 128])
def test_pjds_fp64_matches_oracle(P, oracle_lib, name, make, b):
    A = make()
    x = synth.vector(A.n_cols, seed=11)
    y, _, _ = run_pjds(P, A, x, b=b)
    y_ref, absax, lens = oracle_ref(oracle_lib, A, x)
    r = parity.check_fp64(y, y_ref, absax, lens)
    assert r["ok"], r


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "-".join(f"{k[0]}{v}" for k, v in c.items()))
@pytest.mark.parametrize("name,make", CONFIG_SHAPES, ids=["ragged", "fullrow", "zipf"])
def test_pjds_configs_match_oracle(P, oracle_lib, cfg, name, make):
    A = make()
    x = synth.vector(A.n_cols, seed=12)
    y, _, _ = run_pjds(P, A, x, b=32, cfg=cfg)
    y_ref, absax, lens = oracle_ref(oracle_lib, A, x)
    r = parity.check_fp64(y, y_ref, absax, lens)
    assert r["ok"], r


def test_rows_per_thread_bit_identical_to_one_row(P):
    # R rows per thread only changes the load width, not any row's arithmetic.
    A = synth.zipf_rows(40_000, s=1.7, len_max=300, seed=9)
    x = synth.vector(A.n_cols, seed=9)
    y1, _, _ = run_pjds(P, A, x, cfg=dict(rows_per_thread=1, threads_per_row=1))
    for cfg in (dict(rows_per_thread=2), dict(rows_per_thread=4), dict(threads_per_row=1, unroll=8),
                dict(threads_per_row=1, unroll=16), dict(staged=1), dict(threads_per_row=1, index64=1),
                dict(rows_per_thread=4, index64=1), dict(staged=1, index64=1),
                dict(rows_per_thread=2, unroll=8), dict(rows_per_thread=4, unroll=4)):
        yR, _, _ = run_pjds(P, A, x, cfg=cfg)
        assert np.array_equal(y1.view(np.uint64), yR.view(np.uint64)), cfg


@pytest.mark.parametrize("name,make", SHAPES[:6], ids=[s[0] for s in SHAPES[:6]])
def test_ellr_fp64_matches_oracle_and_pjds_bitwise(P, oracle_lib, name, make):
    A = make()
    x = synth.vector(A.n_cols, seed=13)
    ye = run_ellr(P, A, x)
    y_ref, absax, lens = oracle_ref(oracle_lib, A, x)
    r = parity.check_fp64(ye, y_ref, absax, lens)
    assert r["ok"], r
    # same per-row order and fused multiply-add in both kernels (one thread per row)
    yp, _, _ = run_pjds(P, A, x, cfg=dict(threads_per_row=1))
    assert np.array_equal(ye.view(np.uint64), yp.view(np.uint64))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("b", [32, 256])
def test_staged_kernel_bitwise_and_status(P, dtype, b):
    # the bulk-copy staged kernel does each row's arithmetic exactly like the
    # one-thread-per-row kernel; its bounded waits must all complete
    torch = _torch()
    for A in (synth.hmep_like(n=300_000, seed=31), synth.zipf_rows(70_000, s=1.8, len_max=512, seed=32),
              tiny.random_lengths(1037, 800, max_len=70, seed=3, p_empty=0.15)):
        x = synth.vector(A.n_cols, seed=5)
        P.pjds_device_status(clear=True)
        y1, _, _ = run_pjds(P, A, x, b=b, dtype=dtype, cfg=dict(threads_per_row=1, rows_per_thread=1))
        ys, _, _ = run_pjds(P, A, x, b=b, dtype=dtype, cfg=dict(staged=1))
        assert np.array_equal(y1, ys)
        Hp = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dtype,
                           permute_cols=A.n_rows == A.n_cols)
        Dp = Hp.to_device("cuda")
        xt = torch.from_numpy(x).to("cuda", Dp.vec_dtype)
        ya, yb = (torch.empty(A.n_rows, dtype=Dp.vec_dtype, device="cuda") for _ in range(2))
        P.pjds_spmv_cfg(Dp, xt, ya, threads_per_row=1)
        P.pjds_spmv_cfg(Dp, xt, yb, staged=1)
        torch.cuda.synchronize()
        assert torch.equal(ya, yb)
        assert P.pjds_device_status() == 0


def test_row_sums_exact(P, oracle_lib):
    # x = 1: with one thread per row each fused multiply-add adds val exactly
    # like the oracle's sum, in the same order.
    A = synth.hmep_like(n=200_000, seed=21)
    x = np.ones(A.n_cols)
    y, _, _ = run_pjds(P, A, x, cfg=dict(threads_per_row=1))
    assert np.array_equal(y, oracle_lib.crs_spmv(A, x))


def test_integer_data_exact(P):
    A = tiny.random_lengths(3000, 2000, max_len=100, seed=22, integer_values=True)
    x = np.random.default_rng(3).integers(-3, 4, 2000).astype(np.float64)
    y, _, _ = run_pjds(P, A, x)
    from tests import pins
    assert pins.check_spmv_dense_exact(A, x, y) == []


def test_permuted_basis_roundtrip(P, oracle_lib):
    torch = _torch()
    A = synth.hmep_like(n=150_000, seed=23)
    x = synth.vector(A.n_cols, seed=23)
    y_orig, _, _ = run_pjds(P, A, x)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, permute_cols=True)
    D = H.to_device("cuda")
    xt = torch.from_numpy(x).cuda()
    xp = torch.empty_like(xt)
    yp = torch.empty_like(xt)
    y = torch.empty_like(xt)
    P.pjds_permute(D, xt, xp)
    P.pjds_spmv(D, xp, yp)
    P.pjds_unpermute(D, yp, y)
    torch.cuda.synchronize()
    assert np.array_equal(xp.cpu().numpy(), x[H.perm])
    assert np.array_equal(y.cpu().numpy().view(np.uint64), y_orig.view(np.uint64))
    y_ref, absax, lens = oracle_ref(oracle_lib, A, x)
    assert parity.check_fp64(y.cpu().numpy(), y_ref, absax, lens)["ok"]


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("name,make", [SHAPES[0], SHAPES[5], SHAPES[6]], ids=["banded", "hmep", "zipf"])
def test_reduced_precision_matches_oracle(P, oracle_lib, dtype, name, make):
    A = make()
    x32 = synth.vector(A.n_cols, seed=14).astype(np.float32)
    xd = x32.astype(np.float64)
    y, _, _ = run_pjds(P, A, x32, dtype=dtype, cfg=dict(threads_per_row=1))
    Ar = A._replace(val=oracle_lib.round_f32(A.val) if dtype == "f32" else oracle_lib.round_bf16(A.val))
    y_ref, absax, lens = oracle_ref(oracle_lib, Ar, xd)
    r = parity.check_fp32(y, y_ref, absax, lens)
    assert r["ok"], r
    # R > 1 path for reduced precision (vector loads of 2 or 4 values)
    for R in (2, 4):
        yR, _, _ = run_pjds(P, A, x32, dtype=dtype, cfg=dict(rows_per_thread=R))
        assert np.array_equal(yR, y)
    ye = run_ellr(P, A, x32, dtype=dtype)
    assert np.array_equal(ye, y)


def test_empty_and_degenerate(P):
    torch = _torch()
    # all rows empty: y must be all zeros (no stored entries, no launch)
    A = tiny.from_lengths([0] * 100, 7)
    y, H, _ = run_pjds(P, A, np.ones(7))
    assert H.n_stored == 0 and np.array_equal(y, np.zeros(100))
    ye = run_ellr(P, A, np.ones(7))
    assert np.array_equal(ye, np.zeros(100))
    # zero rows: nothing to do, success
    A0 = tiny.from_lengths([], 3)
    H0 = P.pjds_create(0, 3, A0.row_ptr, A0.col, A0.val)
    D0 = H0.to_device("cuda")
    P.pjds_spmv(D0, torch.zeros(3, dtype=torch.float64, device="cuda"),
                torch.zeros(0, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()


def test_host_entry_point_matches_device_path(P):
    torch = _torch()
    A = synth.banded_uniform(n=20_000, seed=1234)
    x = synth.vector(A.n_cols, seed=15)
    y_dev, H, D = run_pjds(P, A, x)
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty(A.n_rows, dtype=torch.float64).pin_memory()
    xd = torch.empty(A.n_cols, dtype=torch.float64, device="cuda")
    yd = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    P.pjds_spmv_host(D, xh, yh, xd, yd)
    assert np.array_equal(yh.numpy(), y_dev)


def test_stream_argument_is_used(P):
    torch = _torch()
    A = synth.hmep_like(n=50_000, seed=16)
    x = synth.vector(A.n_cols, seed=16)
    y_ref, _, _ = run_pjds(P, A, x)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val)
    D = H.to_device("cuda")
    s = torch.cuda.Stream()
    xt = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        P.pjds_spmv(D, xt, y, stream=s)
    s.synchronize()
    assert np.array_equal(y.cpu().numpy(), y_ref)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("b,permute", [(32, False), (64, True), (256, False)])
def test_tile_order_bitwise_equal_to_sorted_order(P, dtype, b, permute):
    # the traversal table only changes which warp takes which 32-row tile:
    # every kernel that follows it writes the same bits as without it
    torch = _torch()
    for A in (synth.hmep_like(n=150_000, seed=41), synth.zipf_rows(30_000, s=1.8, len_max=400, seed=42),
              tiny.random_lengths(1037, 1037, max_len=70, seed=43, p_empty=0.15)):
        H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dtype, permute_cols=permute)
        Do, Dn = H.to_device("cuda"), H.to_device("cuda", tile_order=False)
        assert Do.struct.tile_order and not Dn.struct.tile_order
        x = torch.from_numpy(synth.vector(A.n_cols, seed=44)).to("cuda", Do.vec_dtype)
        for cfg in (dict(threads_per_row=1), dict(rows_per_thread=2), dict(rows_per_thread=4), dict(threads_per_row=2),
                    dict(threads_per_row=8, block_threads=64), dict(), dict(index64=1), dict(rows_per_thread=2, index64=1)):
            yo = torch.full((A.n_rows,), float("nan"), dtype=Do.vec_dtype, device="cuda")
            yn = torch.full_like(yo, float("nan"))
            P.pjds_spmv_cfg(Do, x, yo, tile_order=1, plan=-1, **cfg)
            P.pjds_spmv_cfg(Dn, x, yn, plan=-1, **cfg)
            torch.cuda.synchronize()
            assert torch.equal(yo.view(torch.int16 if dtype != "f64" else torch.int64),
                               yn.view(torch.int16 if dtype != "f64" else torch.int64)), (cfg, A.n_rows)
        H.destroy()


def test_tile_order_entry_out_of_range_is_skipped(P):
    # an entry outside 0 .. n_pad/32 - 1 is skipped by the kernels' range check:
    # the rows of the tile it replaced are not written, every other row is
    torch = _torch()
    A = synth.hmep_like(n=20_000, seed=45)
    x = synth.vector(A.n_cols, seed=45)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, permute_cols=True)
    D = H.to_device("cuda")
    n_t = H.n_pad // 32
    bad = D.tile_order.clone()
    lost = int(bad[7].item())
    bad[7] = n_t
    D.tile_order = bad
    D.struct.tile_order = bad.data_ptr()
    xt = torch.from_numpy(x[H.perm]).cuda()
    Dn = H.to_device("cuda", tile_order=False)
    skipped = torch.zeros(A.n_rows, dtype=torch.bool, device="cuda")
    skipped[lost * 32:min(lost * 32 + 32, A.n_rows)] = True
    for cfg in (dict(threads_per_row=1), dict(threads_per_row=4), dict(rows_per_thread=2)):
        y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(y)
        P.pjds_spmv_cfg(D, xt, y, tile_order=1, **cfg)
        P.pjds_spmv_cfg(Dn, xt, ref, **cfg)
        torch.cuda.synchronize()
        assert torch.isnan(y[skipped]).all(), cfg
        assert torch.equal(y[~skipped], ref[~skipped]), cfg


@pytest.mark.parametrize("dtype,permute", [("f64", False), ("f32", True), ("bf16", False)])
def test_host_stream_equals_single_products(P, dtype, permute):
    # overlapped host stream: every y_v bit for bit the device product of x_v
    torch = _torch()
    A = synth.hmep_like(n=50_000, seed=61)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype, permute_cols=permute)
    D = H.to_device("cuda")
    n_vec = 5
    xs = [torch.from_numpy(synth.vector(A.n_cols, seed=70 + v)).to(D.vec_dtype).pin_memory() for v in range(n_vec)]
    xs.append(xs[1])  # a host buffer may repeat
    ys = [torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype).pin_memory() for _ in xs]
    xd = [torch.empty(A.n_cols, dtype=D.vec_dtype, device="cuda") for _ in range(2)]
    yd = [torch.empty(A.n_rows, dtype=D.vec_dtype, device="cuda") for _ in range(2)]
    P.pjds_spmv_host_stream(D, xs, ys, xd, yd)
    for v, (xh, yh) in enumerate(zip(xs, ys)):
        ref = torch.empty(A.n_rows, dtype=D.vec_dtype, device="cuda")
        P.pjds_spmv(D, xh.cuda(), ref)
        torch.cuda.synchronize()
        assert torch.equal(ref.cpu(), yh), v
    # one vector, and nothing to do
    y1 = [torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype).pin_memory()]
    P.pjds_spmv_host_stream(D, xs[:1], y1, xd, yd)
    assert torch.equal(y1[0], ys[0])
    P.pjds_spmv_host_stream(D, [], [], xd, yd)


PLAN_SHAPES = [
    ("zipf_wide", lambda: synth.zipf_rows(50_000, s=1.6, len_max=1024, seed=21)),
    ("ragged_long", lambda: tiny.from_lengths([700, 300, 90, 17] + [1, 2, 5, 30] * 300 + [0] * 40, 1500, seed=22)),
    ("one_full_row", lambda: tiny.one_full_row(900, full_row=11)),
    ("ragged_tail", lambda: tiny.random_lengths(1037, 1037, max_len=70, seed=23, p_empty=0.15)),
]


# the permuted basis needs a square matrix: the rectangular shape runs in the original basis only
PLAN_CASES = [(name, make, permute) for name, make in PLAN_SHAPES for permute in (False, True)
              if not (permute and name == "ragged_long")]


@pytest.mark.parametrize("name,make,permute", PLAN_CASES, ids=[f"{c[0]}-{'perm' if c[2] else 'orig'}" for c in PLAN_CASES])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("b", [32, 128])
def test_plan_rows_bit_identical_to_uniform_mappings(P, name, make, permute, dtype, b):
    # each row of the per-tile mapping is summed as the uniform mapping with
    # its tile's lanes per row sums it (one thread per row for kinds 0, 1, 3)
    torch = _torch()
    A = make()
    assert not permute or A.n_rows == A.n_cols
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dtype, permute_cols=permute)
    D = H.to_device("cuda")
    xt = torch.from_numpy(synth.vector(A.n_cols, seed=24)).to(device="cuda", dtype=D.vec_dtype)

    def run(**cfg):
        y = torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
        P.pjds_spmv_cfg(D, xt, y, **cfg)
        torch.cuda.synchronize()
        return y.cpu().numpy()

    y_plan = run(plan=1)
    uniform = {t: run(threads_per_row=t, plan=-1) for t in (1, 2, 4, 8)}
    lanes = np.zeros(H.n_pad, np.int64)
    for _, row0, rows, kind in H.plan:
        lanes[row0:row0 + rows] = 1 if kind in (0, 1, 3) else kind
    assert np.all(lanes[:A.n_rows] > 0)
    out = np.arange(A.n_rows) if permute else H.perm.astype(np.int64)
    want = np.empty_like(y_plan)
    for t in (1, 2, 4, 8):
        rows = out[lanes[:A.n_rows] == t]
        want[rows] = uniform[t][rows]
    assert np.array_equal(y_plan.view(np.uint8), want.view(np.uint8))
    # the default takes the plan exactly when the row lengths are widely
    # spread and the matrix is large enough for its dtype
    spread = H.n_max * A.n_rows > 4 * A.nnz
    big = A.n_rows >= {"f64": 1 << 16, "f32": 1 << 17, "bf16": 1 << 18}[dtype]
    assert P.pjds_spmv_resolve(D)["plan"] == (1 if spread and big else -1)
