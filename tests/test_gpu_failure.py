"""Failure detection on the GPU without a fault: a bounded wait on an mbarrier
that nothing completes gives up, reports its bit through the device status
word, and the context remains usable for the next product."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import pjds
    return torch, pjds


@pytest.mark.parametrize("which,bit", [(0, 1), (1, 2)])
def test_wait_that_runs_out_reports_and_returns(mods, oracle_lib, which, bit):
    torch, pjds = mods
    assert pjds.pjds_device_status(clear=True) in (0, 1, 2, 3)
    t0 = time.perf_counter()
    pjds.pjds_wait_selftest(which)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert waited < 5.0
    assert pjds.pjds_device_status(clear=True) == bit
    assert pjds.pjds_device_status(clear=True) == 0
    # the context still works
    A = synth.hmep_like(n=50_000, seed=3)
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val)
    D = H.to_device("cuda")
    x = synth.vector(A.n_cols, seed=3)
    y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    pjds.pjds_spmv_cfg(D, torch.from_numpy(x).cuda(), y, staged=1)
    torch.cuda.synchronize()
    yr = oracle_lib.crs_spmv(A, x)
    assert np.max(np.abs(y.cpu().numpy() - yr)) <= 1e-14 * np.max(oracle_lib.crs_absmv(A, x))
    assert pjds.pjds_device_status() == 0
