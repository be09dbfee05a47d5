"""GPU parity of the pattern product y = S x (pjds_spmv_pattern), S the
sparsity pattern of A: the product's column stream, x gathers and y stores
without the value stream, used as the gather ceiling of the product.

Against the oracle's CRS product of the same pattern with every value 1: the
oracle forms 1 * x[c] exactly and adds in CRS order, the kernel adds x[c] in
the same order, so fp64 results are equal bit for bit.
"""
import numpy as np
import pytest

import synth
from synth import Crs, tiny
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


def _ones(A):
    return Crs(A.n_rows, A.n_cols, A.row_ptr, A.col, np.ones(A.nnz))


SHAPES = [
    ("ragged_tail", lambda: tiny.random_lengths(1037, 800, max_len=70, seed=3, p_empty=0.15)),
    ("one_full_row", lambda: tiny.one_full_row(700, full_row=500)),
    ("hmep_small", lambda: synth.hmep_like(n=100_000, seed=7)),
    ("hmep_1M", lambda: synth.hmep_like(n=1_100_000, seed=5)),
    ("zipf", lambda: synth.zipf_rows(60_000, s=2.0, len_max=512, seed=8)),
    ("single", lambda: tiny.from_lengths([3], 5, seed=2)),
]
# one thread per row (the pattern product's mappings); small matrices would
# otherwise default to several threads per row
CFGS = [dict(threads_per_row=1), dict(threads_per_row=1, tile_order=-1), dict(threads_per_row=1, tile_order=1),
        dict(threads_per_row=1, unroll=8), dict(threads_per_row=1, unroll=16, block_threads=128),
        dict(threads_per_row=1, index64=1), dict(rows_per_thread=2), dict(rows_per_thread=4, tile_order=1),
        dict(rows_per_thread=2, unroll=8, index64=1)]


@pytest.mark.parametrize("cfg", CFGS, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
@pytest.mark.parametrize("name,make", SHAPES, ids=[s[0] for s in SHAPES])
def test_pattern_fp64_bitwise_equals_oracle(P, oracle_lib, name, make, cfg):
    import torch
    A = make()
    x = synth.vector(A.n_cols, seed=21)
    D = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64").to_device("cuda")
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    P.pjds_spmv_pattern(D, torch.from_numpy(x).cuda(), y, **cfg)
    torch.cuda.synchronize()
    want = oracle_lib.crs_spmv(_ones(A), x)
    got = y.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), int(np.sum(got != want))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_pattern_fp32_vectors_within_bound(P, oracle_lib, dtype):
    import torch
    A = synth.hmep_like(n=200_000, seed=9)
    x = synth.vector(A.n_cols, seed=22).astype(np.float32)
    D = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype).to_device("cuda")
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float32, device="cuda")
    P.pjds_spmv_pattern(D, torch.from_numpy(x).cuda(), y, threads_per_row=1)
    torch.cuda.synchronize()
    S = _ones(A)
    xd = x.astype(np.float64)
    r = parity.check_fp32(y.cpu().numpy(), oracle_lib.crs_spmv(S, xd), oracle_lib.crs_absmv(S, xd),
                          np.diff(A.row_ptr))
    assert r["ok"], r


def test_pattern_permuted_basis(P, oracle_lib):
    import torch
    A = synth.hmep_like(n=50_000, seed=4)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64", permute_cols=True)
    perm = H.perm.copy()
    D = H.to_device("cuda")
    x = synth.vector(A.n_cols, seed=23)
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    P.pjds_spmv_pattern(D, torch.from_numpy(x[perm]).cuda(), y, threads_per_row=1)
    torch.cuda.synchronize()
    want = oracle_lib.crs_spmv(_ones(A), x)[perm]
    assert np.array_equal(y.cpu().numpy().view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("cfg", [dict(plan=1), dict(threads_per_row=2), dict(threads_per_row=8, unroll=2)])
@pytest.mark.parametrize("dtype", ["f64", "bf16"])
def test_pattern_plan_and_lanes_within_bound(P, oracle_lib, cfg, dtype):
    # several lanes per row change the summation order: the oracle's bound
    import torch
    A = synth.zipf_rows(70_000, s=2.0, len_max=512, seed=8)
    D = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype).to_device("cuda")
    x = synth.vector(A.n_cols, seed=25)
    xd = x.astype(np.float32).astype(np.float64) if dtype != "f64" else x
    y = torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
    P.pjds_spmv_pattern(D, torch.from_numpy(xd).to("cuda", D.vec_dtype), y, **cfg)
    torch.cuda.synchronize()
    S = _ones(A)
    check = parity.check_fp64 if dtype == "f64" else parity.check_fp32
    r = check(y.double().cpu().numpy(), oracle_lib.crs_spmv(S, xd), oracle_lib.crs_absmv(S, xd), np.diff(A.row_ptr))
    assert r["ok"], r


def test_pattern_batch_within_bound(P, oracle_lib):
    import torch
    from paper_1112_5588_gb300 import batch
    mats = [synth.zipf_rows(n, s=2.0, len_max=300, seed=30 + n % 7) for n in (20_000, 70_001, 5_003)]
    devs = [P.pjds_create(M.n_rows, M.n_cols, M.row_ptr, M.col, M.val, b=32).to_device("cuda") for M in mats]
    xs = [synth.vector(M.n_cols, seed=26 + k) for k, M in enumerate(mats)]
    ys = [torch.full((M.n_rows,), float("nan"), dtype=torch.float64, device="cuda") for M in mats]
    B = batch.Batch(devs, [torch.from_numpy(x).cuda() for x in xs], ys)
    B.run_pattern()
    torch.cuda.synchronize()
    for M, x, y in zip(mats, xs, ys):
        S = _ones(M)
        r = parity.check_fp64(y.cpu().numpy(), oracle_lib.crs_spmv(S, x), oracle_lib.crs_absmv(S, x),
                              np.diff(M.row_ptr))
        assert r["ok"], r
    B.destroy()


@pytest.mark.parametrize("cfg", [dict(staged=1)])
def test_pattern_rejects_other_mappings(P, cfg):
    import torch
    A = synth.zipf_rows(70_000, s=2.0, len_max=512, seed=8)
    D = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64").to_device("cuda")
    x = torch.zeros(A.n_cols, dtype=torch.float64, device="cuda")
    y = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PjdsError):
        P.pjds_spmv_pattern(D, x, y, **cfg)


@pytest.mark.parametrize("k", [2, 8, 32])
def test_pattern_spmm_bitwise_equals_oracle(P, oracle_lib, k):
    import torch
    from paper_1112_5588_gb300 import batch
    A = synth.block_dense(n_brow=2_000, bs=4, nb=36, frac=0.05, seed=3)
    D = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64").to_device("cuda")
    X = np.random.default_rng(k).uniform(-1, 1, (A.n_cols, k))
    Y = torch.full((A.n_rows, k), float("nan"), dtype=torch.float64, device="cuda")
    batch.spmm_pattern(D, torch.from_numpy(X).cuda(), Y)
    torch.cuda.synchronize()
    want = oracle_lib.crs_spmm(_ones(A), X)
    got = Y.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
