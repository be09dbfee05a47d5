"""GPU parity at full size, in the launch configuration the benchmark times.

HMEp-like N = 6.2M (~93M nonzeros) and the 27-point stencil on 165^3
(N = 4.49M, ~108M nonzeros). The fp64 oracle evaluates every row (OpenMP on
the host), so every output element is compared.
"""
import numpy as np
import pytest

import synth
from tests import parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds
    return pjds


@pytest.fixture(scope="module")
def hmep():
    return synth.hmep_like(n=6_200_000, seed=1234)


@pytest.fixture(scope="module")
def stencil():
    return synth.stencil27(g=165, p_drop=0.1, seed=1234)


def _spmv(P, A, x, dtype="f64", fmt="pjds", cfg=None):
    import torch
    if fmt == "pjds":
        H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype)
    else:
        H = P.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype=dtype)
    D = H.to_device("cuda")
    H.destroy()
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=D.vec_dtype)
    y = torch.full((A.n_rows,), float("nan"), dtype=D.vec_dtype, device="cuda")
    if cfg:
        P.pjds_spmv_cfg(D, xt, y, **cfg)
    else:
        (P.pjds_spmv if fmt == "pjds" else P.ellr_spmv)(D, xt, y)
    torch.cuda.synchronize()
    out = y.cpu().numpy().astype(np.float64)
    del D, xt, y
    torch.cuda.empty_cache()
    return out


@pytest.mark.parametrize("fmt", ["pjds", "ellr"])
def test_hmep_fp64_full(P, oracle_lib, hmep, fmt):
    x = synth.vector(hmep.n_cols, seed=1)
    y = _spmv(P, hmep, x, fmt=fmt)
    r = parity.check_fp64(y, oracle_lib.crs_spmv(hmep, x), oracle_lib.crs_absmv(hmep, x), np.diff(hmep.row_ptr))
    assert r["ok"], r


def test_hmep_fp64_staged_full(P, oracle_lib, hmep):
    x = synth.vector(hmep.n_cols, seed=1)
    P.pjds_device_status(clear=True)
    y = _spmv(P, hmep, x, cfg=dict(staged=1))
    r = parity.check_fp64(y, oracle_lib.crs_spmv(hmep, x), oracle_lib.crs_absmv(hmep, x), np.diff(hmep.row_ptr))
    assert r["ok"], r
    assert P.pjds_device_status() == 0


def test_hmep_fp32_full(P, oracle_lib, hmep):
    x32 = synth.vector(hmep.n_cols, seed=2).astype(np.float32)
    y = _spmv(P, hmep, x32, dtype="f32")
    Ar = hmep._replace(val=oracle_lib.round_f32(hmep.val))
    xd = x32.astype(np.float64)
    r = parity.check_fp32(y, oracle_lib.crs_spmv(Ar, xd), oracle_lib.crs_absmv(Ar, xd), np.diff(hmep.row_ptr))
    assert r["ok"], r


def test_stencil_fp64_full(P, oracle_lib, stencil):
    x = synth.vector(stencil.n_cols, seed=3)
    y = _spmv(P, stencil, x)
    r = parity.check_fp64(y, oracle_lib.crs_spmv(stencil, x), oracle_lib.crs_absmv(stencil, x),
                          np.diff(stencil.row_ptr))
    assert r["ok"], r


def test_stencil_bf16_full(P, oracle_lib, stencil):
    x32 = synth.vector(stencil.n_cols, seed=4).astype(np.float32)
    y = _spmv(P, stencil, x32, dtype="bf16")
    Ar = stencil._replace(val=oracle_lib.round_bf16(stencil.val))
    xd = x32.astype(np.float64)
    r = parity.check_fp32(y, oracle_lib.crs_spmv(Ar, xd), oracle_lib.crs_absmv(Ar, xd), np.diff(stencil.row_ptr))
    assert r["ok"], r
