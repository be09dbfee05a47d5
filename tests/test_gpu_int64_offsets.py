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

Needs about 50 GB of free host memory and 32 GB of free device memory;
skipped otherwise.
"""
import numpy as np
import pytest

from synth import Crs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 1 << 24
STRIDE = 4099  # column step between a row's entries; 132 * 4099 < N keeps them distinct


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


def _mem_available_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 1e6
    except OSError:
        pass
    return 0.0


@pytest.fixture(scope="module")
def big():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    if _mem_available_gb() < 80:
        pytest.skip("needs about 50 GB of free host memory")
    if torch.cuda.mem_get_info()[0] < 48e9:
        pytest.skip("needs about 32 GB of free device memory")
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds

    r_all = np.arange(N, dtype=np.int64)
    row_ptr = np.zeros(N + 1, np.int64)
    np.cumsum(_lengths(r_all), out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float64)
    step = 1 << 18
    for s in range(0, N, step):
        e = min(s + step, N)
        c, v = _entries(r_all[s:e])
        col[row_ptr[s]:row_ptr[e]] = c
        val[row_ptr[s]:row_ptr[e]] = v
    H = pjds.pjds_create(N, N, row_ptr, col, val, b=32, dtype="bf16")
    assert H.n_stored + H.n_pad > 2**31
    D = H.to_device("cuda")
    H.destroy()
    He = pjds.ellr_create(N, N, row_ptr, col, val, dtype="bf16")
    assert He.n_stored > 2**31
    E = He.to_device("cuda")
    He.destroy()
    del col, val
    x = torch.from_numpy(_x()).cuda()
    yield pjds, D, E, x, row_ptr
    del D, E, x
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
    pjds, D, E, x, _ = big
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
