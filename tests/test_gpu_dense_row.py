"""GPU parity at the longest row: one fully dense row of 2^20 + 37 entries.

The pJDS worst case of Sect. 2.1 (one full row pads its whole block) at a size
where the row alone holds more entries than the rest of the matrix: 50,000 rows,
2^20 + 37 columns, row 123 dense, every other row 0-16 entries. Values are
integers in [-3, 3] and x holds integers in [-4, 4], so every partial sum of
any row is an integer of magnitude at most 12 * (2^20 + 37) < 2^24: exact in
fp32 and fp64 whatever the summation order, and bf16 holds the values exactly.
Every mapping (one thread per row, 2 and 4 rows per thread, 2-8 threads per
row, the per-tile mapping, the staged kernel, both tile orders), the pattern
product and the block product must therefore equal the oracle bit for bit.
"""
import numpy as np
import pytest

from synth import Crs

pytestmark = pytest.mark.gpu

N_ROWS = 50_000
N_COLS = (1 << 20) + 37
DENSE = 123

CONFIGS = [None, dict(threads_per_row=1), dict(threads_per_row=2), dict(threads_per_row=4),
           dict(threads_per_row=8), dict(rows_per_thread=2), dict(rows_per_thread=4), dict(tile_order=1),
           dict(tile_order=-1, threads_per_row=8), dict(plan=1), dict(staged=1)]


def _matrix() -> Crs:
    rng = np.random.default_rng(2026)
    lens = rng.integers(0, 17, size=N_ROWS)
    lens[DENSE] = N_COLS
    row_ptr = np.zeros(N_ROWS + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    col = np.empty(int(row_ptr[-1]), np.int32)
    for i in range(N_ROWS):
        a, e = row_ptr[i], row_ptr[i + 1]
        if i == DENSE:
            col[a:e] = np.arange(N_COLS, dtype=np.int32)
        elif e > a:
            col[a:e] = np.sort(rng.choice(N_COLS, size=e - a, replace=False))
    val = rng.integers(-3, 4, size=len(col)).astype(np.float64)
    return Crs(N_ROWS, N_COLS, row_ptr, col, val)


@pytest.fixture(scope="module")
def case(oracle_lib):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds
    A = _matrix()
    x = np.random.default_rng(7).integers(-4, 5, size=N_COLS).astype(np.float64)
    y_ref = oracle_lib.crs_spmv(A, x)
    assert np.max(np.abs(oracle_lib.crs_absmv(A, np.abs(x)))) < 2 ** 24
    return torch, pjds, A, x, y_ref


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("b", [32, 64])
def test_dense_row_every_mapping_exact(case, dtype, b):
    torch, pjds, A, x, y_ref = case
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dtype)
    assert H.n_max == N_COLS and H.n_stored >= b * N_COLS
    D = H.to_device("cuda")
    xt = torch.from_numpy(x).to("cuda", D.vec_dtype)
    y = torch.empty(N_ROWS, dtype=D.vec_dtype, device="cuda")
    for cfg in CONFIGS:
        y.fill_(float("nan"))
        if cfg is None:
            pjds.pjds_spmv(D, xt, y)
        else:
            pjds.pjds_spmv_cfg(D, xt, y, **cfg)
        torch.cuda.synchronize()
        got = y.double().cpu().numpy()
        assert np.array_equal(got, y_ref), (dtype, b, cfg, int(np.sum(got != y_ref)))
    assert pjds.pjds_device_status(clear=True) == 0


def test_dense_row_pattern_and_block_product_exact(case, oracle_lib):
    torch, pjds, A, x, y_ref = case
    from paper_1112_5588_gb300 import batch
    D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64").to_device("cuda")
    xt = torch.from_numpy(x).to("cuda")
    y = torch.full((N_ROWS,), float("nan"), dtype=torch.float64, device="cuda")
    pjds.pjds_spmv_pattern(D, xt, y)
    torch.cuda.synchronize()
    ones = A._replace(val=np.ones_like(A.val))
    assert np.array_equal(y.cpu().numpy(), oracle_lib.crs_spmv(ones, x))
    X = np.stack([x, -x[::-1].copy(), np.roll(x, 5), np.ones_like(x)], axis=1)
    Y = torch.full((N_ROWS, 4), float("nan"), dtype=torch.float64, device="cuda")
    batch.spmm(D, torch.from_numpy(np.ascontiguousarray(X)).to("cuda"), Y)
    torch.cuda.synchronize()
    assert np.array_equal(Y.cpu().numpy(), oracle_lib.crs_spmm(A, X))
