"""GPU parity of the window mapping (pjds_dev.win_ptr): one CTA per window of
original rows, band intervals of x and the window's y in shared memory.

Each thread runs one sorted row exactly as the one-thread-per-row mapping
does, so every result must equal that mapping's bit for bit, and lie within
the oracle bounds of tests/parity.py. The pattern product over the window
mapping equals the oracle's product with unit values bit for bit.
"""
import numpy as np
import pytest

import synth
from synth import Crs
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


SHAPES = [
    ("hmep_100k", lambda: synth.hmep_like(n=100_000, seed=7)),
    ("hmep_1.1M", lambda: synth.hmep_like(n=1_100_000, seed=5)),
    ("stencil_g41", lambda: synth.stencil27(g=41, p_drop=0.1, seed=3)),
    ("banded_70k", lambda: synth.banded_uniform(n=70_000, hw=40, seed=2)),
]


def _run(P, D, x, **cfg):
    import torch
    y = torch.full((D.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
    P.pjds_spmv_cfg(D, x, y, **cfg)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("name,make", SHAPES, ids=[s[0] for s in SHAPES])
def test_window_bitwise_equals_one_thread_per_row(P, oracle_lib, name, make, dtype):
    import torch
    A = make()
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype)
    assert H.n_win > 0, "a band matrix of at least 2^16 rows has a window plan"
    D = H.to_device("cuda")
    x = synth.vector(A.n_cols, seed=31)
    xt = torch.from_numpy(x).to("cuda", D.vec_dtype)
    y_w = _run(P, D, xt, window=1)
    assert P.pjds_spmv_resolve(D, window=1)["window"] == 1
    y_1 = _run(P, D, xt, rows_per_thread=1, threads_per_row=1, tile_order=1)
    assert not torch.isnan(y_w).any()
    assert torch.equal(y_w.view(torch.int32 if dtype != "f64" else torch.int64),
                       y_1.view(torch.int32 if dtype != "f64" else torch.int64))
    for cfg in (dict(window=1, unroll=8), dict(window=1, index64=1)):
        assert torch.equal(_run(P, D, xt, **cfg), y_w), cfg
    if dtype == "f64":
        y_ref, absax = oracle_lib.crs_spmv(A, x), oracle_lib.crs_absmv(A, x)
        r = parity.check_fp64(y_w.cpu().numpy(), y_ref, absax, np.diff(A.row_ptr))
        assert r["ok"], r


def test_window_is_the_default_for_band_matrices(P, oracle_lib):
    import torch
    A = synth.hmep_like(n=300_000, seed=11)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64")
    D = H.to_device("cuda")
    assert P.pjds_spmv_resolve(D)["window"] == 1
    x = synth.vector(A.n_cols, seed=32)
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    P.pjds_spmv(D, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    r = parity.check_fp64(y.cpu().numpy(), oracle_lib.crs_spmv(A, x), oracle_lib.crs_absmv(A, x),
                          np.diff(A.row_ptr))
    assert r["ok"], r
    # uploaded without the window plan: the uniform mapping, same bits
    D0 = H.to_device("cuda", window=False)
    assert P.pjds_spmv_resolve(D0)["window"] == -1
    y0 = torch.full_like(y, float("nan"))
    P.pjds_spmv(D0, torch.from_numpy(x).cuda(), y0)
    torch.cuda.synchronize()
    assert torch.equal(y.view(torch.int64), y0.view(torch.int64))


def test_window_pattern_product_bitwise_equals_oracle(P, oracle_lib):
    import torch
    A = synth.hmep_like(n=500_000, seed=13)
    D = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64").to_device("cuda")
    x = synth.vector(A.n_cols, seed=33)
    y = torch.full((A.n_rows,), float("nan"), dtype=torch.float64, device="cuda")
    P.pjds_spmv_pattern(D, torch.from_numpy(x).cuda(), y, window=1)
    torch.cuda.synchronize()
    want = oracle_lib.crs_spmv(Crs(A.n_rows, A.n_cols, A.row_ptr, A.col, np.ones(A.nnz)), x)
    got = y.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), int(np.sum(got != want))


def test_window_b64_and_ragged_tail(P, oracle_lib):
    # b = 64 (two tiles per block) and a row count that is not a multiple of
    # the window size or of 32
    import torch
    A = synth.hmep_like(n=200_003, seed=17)
    D = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=64, dtype="f64").to_device("cuda")
    x = synth.vector(A.n_cols, seed=34)
    xt = torch.from_numpy(x).cuda()
    y_w = _run(P, D, xt, window=1)
    y_1 = _run(P, D, xt, rows_per_thread=1, threads_per_row=1)
    assert torch.equal(y_w.view(torch.int64), y_1.view(torch.int64))
    r = parity.check_fp64(y_w.cpu().numpy(), oracle_lib.crs_spmv(A, x), oracle_lib.crs_absmv(A, x),
                          np.diff(A.row_ptr))
    assert r["ok"], r
