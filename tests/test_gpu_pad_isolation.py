"""GPU: padding entries never touch x (Listing 2 stops at a row's own length).

pJDS pads every row of a block to the block's longest row (Sect. 2.1), and the
kernels loop to the block length, so each pad must be skipped, not multiplied:
0 * x[c] would turn a NaN or an infinity in x into a NaN in y. Here x holds NaN
at every column no row references (most of them: the matrices reference at
most a third of their columns) and finite values elsewhere; every product must then
equal the oracle's product with those entries of x set to 0, within the fp64
or fp32 parity bounds, with no NaN anywhere in y. Covered: every uniform
mapping, the per-tile mapping, the staged kernel, the pattern product,
ELLPACK-R, the block product and the batched launch.
"""
import numpy as np
import pytest

import synth
from synth import tiny
from tests import parity

pytestmark = pytest.mark.gpu

CONFIGS = [None, dict(threads_per_row=1), dict(threads_per_row=2), dict(threads_per_row=8),
           dict(rows_per_thread=2), dict(rows_per_thread=4), dict(tile_order=1), dict(tile_order=-1),
           dict(plan=1), dict(staged=1)]


def _spread(A, f):
    """The same rows with column c renamed f*c + 1: most columns unreferenced."""
    return A._replace(n_cols=A.n_cols * f + 1, col=(A.col.astype(np.int64) * f + 1).astype(np.int32))


SHAPES = [("ragged", lambda: tiny.random_lengths(1037, 400_000, max_len=70, seed=91, p_empty=0.2)),
          ("zipf", lambda: _spread(synth.zipf_rows(30_000, s=1.8, len_max=400, seed=92), 5)),
          ("banded", lambda: _spread(synth.banded_uniform(n=20_000, seed=93), 3))]


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import batch, pjds
    return torch, pjds, batch


def _poisoned_x(A, seed):
    """(x with NaN at unreferenced columns, the same x with 0 there)."""
    x = synth.vector(A.n_cols, seed=seed)
    used = np.zeros(A.n_cols, bool)
    used[A.col] = True
    assert (~used).sum() > 0
    return np.where(used, x, np.nan), np.where(used, x, 0.0)


def _ref(oracle_lib, A, x0, dtype):
    if dtype == "f64":
        return A, oracle_lib.crs_spmv(A, x0), oracle_lib.crs_absmv(A, x0), parity.check_fp64
    Ar = A._replace(val=oracle_lib.round_f32(A.val) if dtype == "f32" else oracle_lib.round_bf16(A.val))
    xr = x0.astype(np.float32).astype(np.float64)
    return Ar, oracle_lib.crs_spmv(Ar, xr), oracle_lib.crs_absmv(Ar, xr), parity.check_fp32


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("name,make", SHAPES, ids=[s[0] for s in SHAPES])
def test_pads_never_read_x(mods, oracle_lib, dtype, name, make):
    torch, pjds, batch = mods
    A = make()
    xn, x0 = _poisoned_x(A, seed=5)
    Ar, y_ref, absax, check = _ref(oracle_lib, A, x0, dtype)
    lens = np.diff(A.row_ptr)
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype)
    assert H.n_stored > H.nnz  # there are pads to skip
    D = H.to_device("cuda")
    xt = torch.from_numpy(xn).to("cuda", D.vec_dtype)
    y = torch.empty(A.n_rows, dtype=D.vec_dtype, device="cuda")
    for cfg in CONFIGS:
        y.fill_(float("nan"))
        if cfg is None:
            pjds.pjds_spmv(D, xt, y)
        else:
            pjds.pjds_spmv_cfg(D, xt, y, **cfg)
        torch.cuda.synchronize()
        got = y.double().cpu().numpy()
        assert not np.isnan(got).any(), (cfg, int(np.isnan(got).sum()))
        r = check(got, y_ref, absax, lens)
        assert r["ok"], (cfg, r)
    assert pjds.pjds_device_status(clear=True) == 0
    # the pattern product: pads skipped the same way
    pjds.pjds_spmv_pattern(D, xt, y)
    torch.cuda.synchronize()
    got = y.double().cpu().numpy()
    assert not np.isnan(got).any()
    xr = x0 if dtype == "f64" else x0.astype(np.float32).astype(np.float64)
    ones = A._replace(val=np.ones_like(A.val))
    r = check(got, oracle_lib.crs_spmv(ones, xr), oracle_lib.crs_absmv(ones, xr), lens)
    assert r["ok"], r
    # ELLPACK-R pads its rows to the longest row of the matrix
    E = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype=dtype).to_device("cuda")
    y.fill_(float("nan"))
    pjds.ellr_spmv(E, xt, y)
    torch.cuda.synchronize()
    got = y.double().cpu().numpy()
    assert not np.isnan(got).any()
    assert check(got, y_ref, absax, lens)["ok"]


@pytest.mark.parametrize("dtype,k", [("f64", 4), ("f32", 8), ("bf16", 4)])
def test_pads_never_read_x_block_and_batched(mods, oracle_lib, dtype, k):
    torch, pjds, batch = mods
    mats = [make() for _, make in SHAPES]
    Ds, xs, ys, refs = [], [], [], []
    for m, A in enumerate(mats):
        xn, x0 = _poisoned_x(A, seed=20 + m)
        Ar, y_ref, absax, check = _ref(oracle_lib, A, x0, dtype)
        D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype).to_device("cuda")
        Ds.append(D)
        xs.append(torch.from_numpy(xn).to("cuda", D.vec_dtype))
        ys.append(torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda"))
        refs.append((y_ref, absax, check, np.diff(A.row_ptr)))
        # block product: the poisoned columns of X are NaN in every right-hand side
        X0 = np.stack([x0 * (c + 1) for c in range(k)], axis=1)
        Xn = np.where(np.isnan(xn)[:, None], np.nan, X0)
        Y = torch.full((A.n_rows, k), float("nan"), dtype=D.vec_dtype, device="cuda")
        batch.spmm(D, torch.from_numpy(np.ascontiguousarray(Xn)).to("cuda", D.vec_dtype), Y)
        torch.cuda.synchronize()
        got = Y.double().cpu().numpy()
        assert not np.isnan(got).any(), (m, int(np.isnan(got).sum()))
        Xr = X0 if dtype == "f64" else X0.astype(np.float32).astype(np.float64)
        Yr = oracle_lib.crs_spmm(Ar, Xr)
        S = oracle_lib.crs_spmm(Ar._replace(val=np.abs(Ar.val)), np.abs(Xr))
        for c in range(k):
            assert check(got[:, c], Yr[:, c], S[:, c], np.diff(A.row_ptr))["ok"], (m, c)
    B = batch.Batch(Ds, xs, ys)
    B.run()
    torch.cuda.synchronize()
    for m, (y_ref, absax, check, lens) in enumerate(refs):
        got = ys[m].double().cpu().numpy()
        assert not np.isnan(got).any(), m
        assert check(got, y_ref, absax, lens)["ok"], m
