"""GPU parity beyond 2^31 stored elements: the 64-bit offset kernels at their real size.

A matrix of 2^24 rows with 128-132 entries each (2.18G nonzeros, 2.21G stored
in ELLPACK-R) puts element offsets col_start[j] + i beyond 2^31 on every row
of 129 entries or more, so the launchers take the 64-bit index instances
without being told to. Values are multiples of 1/8 in [-7/8, 7/8] (exact in
bf16) and x holds multiples of 1/16 in [-1/2, 1/2]: every product is a
multiple of 1/128 and every partial sum stays below 64 in magnitude, so the
fp32 accumulation of the bf16 kernels is exact, and sampled rows must equal
the fp64 oracle bit for bit. Rows and columns come from closed formulas, so
the oracle evaluates the sampled rows without the full matrix.

The matrix never exists on the host: pjds_create_shape gives the pJDS
structure from the row lengths (2^24 + 1 offsets), and the test fills col
and val in device memory one jagged diagonal at a time from the same
formulas; ELLPACK-R is filled on the device the same way. About 28 GB of
device memory and a few hundred MB of host memory.
"""
import numpy as np
import pytest

from synth import Crs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 1 << 24
STRIDE = 4099  # column step between a row's entries; 132 * 4099 < N keeps them distinct
N_MAX = 132


def _lengths(r):
    return 128 + ((r ^ (r >> 3)) % 5)


def _entries(rows):
    """Columns and values of the given rows (int64 array), concatenated in CRS order."""
    lens = _lengths(rows)
    reps = np.repeat(rows, lens)
    k = np.arange(int(lens.sum()), dtype=np.int64) - np.repeat(np.cumsum(lens) - lens, lens)
    col = ((reps + k * STRIDE) % N).astype(np.int32)
    val = (((reps * 3 + k * 5) % 15) - 7) * 0.125
    return col, val


def _x():
    j = np.arange(N, dtype=np.int64)
    return ((((j * 11) % 17) - 8) / 16.0).astype(np.float32)


def _diagonal(torch, r, j):
    """Entry j of original rows r (int64 device tensor): (column, bf16 bits), pads (-1, +0)."""
    live = j < _lengths(r)
    c = torch.where(live, (r + j * STRIDE) % N, torch.full_like(r, -1)).to(torch.int32)
    v = torch.where(live, (((r * 3 + j * 5) % 15) - 7).to(torch.float32) * 0.125, torch.zeros((), device=r.device))
    return c, v.to(torch.bfloat16).view(torch.int16)


class _EllrView:
    """The few attributes ellr_spmv reads, over caller-filled device arrays."""

    def __init__(self, P, torch, row_max, col, val, nnz):
        self.n_rows = self.n_cols = self.n_pad = N
        self.n_max = N_MAX
        self.vec_dtype = torch.float32
        self._keep = (row_max, col, val)
        s = P._EllrDevS()
        s.n_rows, s.n_cols, s.n_pad, s.n_max = N, N, N, N_MAX
        s.nnz, s.n_stored, s.dtype = nnz, N * N_MAX, 2
        s.row_max, s.col, s.val = row_max.data_ptr(), col.data_ptr(), val.data_ptr()
        self.struct = s


@pytest.fixture(scope="module")
def big():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    if torch.cuda.mem_get_info()[0] < 40e9:
        pytest.skip("needs about 30 GB of free device memory")
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds

    r_all = np.arange(N, dtype=np.int64)
    row_ptr = np.zeros(N + 1, np.int64)
    np.cumsum(_lengths(r_all), out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    S = pjds.pjds_create_shape(N, N, row_ptr, b=32, dtype="bf16")
    assert S.n_stored + S.n_pad > 2**31 and S.n_max == N_MAX
    cs = S.col_start.copy()
    perm = torch.from_numpy(S.perm.astype(np.int64)).cuda()
    col = torch.empty(S.n_stored, dtype=torch.int32, device="cuda")
    val = torch.empty(S.n_stored, dtype=torch.int16, device="cuda")
    for j in range(S.n_max):
        a, e = int(cs[j]), int(cs[j + 1])
        col[a:e], val[a:e] = _diagonal(torch, perm[: e - a], j)
    del perm
    D = pjds.PjdsDevice(S, "cuda", col=col, val=val)
    S.destroy()
    # ELLPACK-R: entry j of row i at j * N + i
    rows = torch.arange(N, dtype=torch.int64, device="cuda")
    ecol = torch.empty(N * N_MAX, dtype=torch.int32, device="cuda")
    eval_ = torch.empty(N * N_MAX, dtype=torch.int16, device="cuda")
    for j in range(N_MAX):
        ecol[j * N:(j + 1) * N], eval_[j * N:(j + 1) * N] = _diagonal(torch, rows, j)
    E = _EllrView(pjds, torch, _lengths(rows).to(torch.int32), ecol, eval_, nnz)
    del rows
    x = torch.from_numpy(_x()).cuda()
    torch.cuda.synchronize()
    yield pjds, D, E, x
    del D, E, x, col, val, ecol, eval_
    torch.cuda.empty_cache()


def _sample_rows():
    rng = np.random.default_rng(2024)
    rows = np.concatenate([[0, 1, 2, N - 2, N - 1], rng.integers(0, N, 4096)]).astype(np.int64)
    # rows of the longest class (132 entries) reach the largest offsets
    long_rows = np.nonzero(_lengths(np.arange(4096, dtype=np.int64)) == 132)[0]
    return np.unique(np.concatenate([rows, long_rows, N - 4096 + long_rows]))


def _oracle_rows(oracle_lib, rows):
    lens = _lengths(rows)
    rp = np.zeros(len(rows) + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    col, val = _entries(rows)
    return oracle_lib.crs_spmv(Crs(len(rows), N, rp, col, val), _x().astype(np.float64))


@pytest.mark.parametrize("cfg", [None, dict(rows_per_thread=1), dict(threads_per_row=4), dict(tile_order=-1),
                                 dict(staged=1), dict(plan=1), "ellr"])
def test_offsets_beyond_2_31_exact(big, oracle_lib, cfg):
    import torch
    pjds, D, E, x = big
    y = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
    if cfg == "ellr":
        pjds.ellr_spmv(E, x, y)
    elif cfg is None:
        assert pjds.pjds_spmv_resolve(D)["index64"] == 0  # 64-bit offsets come from the size, not the flag
        pjds.pjds_spmv(D, x, y)
    else:
        pjds.pjds_spmv_cfg(D, x, y, **cfg)
    torch.cuda.synchronize()
    if cfg == dict(staged=1):
        assert pjds.pjds_device_status(clear=True) == 0
    rows = _sample_rows()
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
    want = _oracle_rows(oracle_lib, rows)
    assert np.array_equal(got, want), (cfg, int(np.sum(got != want)))
    assert not torch.isnan(y).any()
