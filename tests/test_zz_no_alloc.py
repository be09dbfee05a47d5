"""pjds_cg_solve_static — the CG solve for callers that cannot allocate device
memory (it uses the library's static device workspace instead of one the
caller passes) — checked through the C ABI against pjds_cg_solve, which takes
a caller workspace, on two calls in a row (the static array keeps the first
call's contents when the second starts).

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test.
"""
import ctypes

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
    from paper_1112_5588_gb300 import krylov, pjds
    return torch, pjds, krylov


def _dev(pjds, A, dtype):
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype, permute_cols=True)
    return H.to_device("cuda"), H.perm.copy()


@pytest.mark.parametrize("lo", [None, "f32"])
def test_static_workspace_matches_caller_workspace_twice(mods, oracle_lib, lo):
    torch, pjds, krylov = mods
    A = synth.stencil27(g=20, p_drop=0.1, seed=7)      # 8000 rows
    D64, perm = _dev(pjds, A, "f64")
    Dlo = _dev(pjds, A, lo)[0] if lo else None
    lib = krylov._lib
    for call, seed in enumerate((3, 4)):  # two calls in a row, different right-hand sides
        b = synth.vector(A.n_rows, seed=seed)
        bp = torch.from_numpy(b[perm]).cuda()
        x_ref = torch.zeros_like(bp)
        x_st = torch.zeros_like(bp)
        ref = krylov.cg_solve(D64, Dlo, bp, x_ref, max_outer=6, inner_iters=50)
        # use_graph = 1 is passed on purpose: the entry point ignores it and
        # launches the inner steps directly, creating no graph
        o = krylov._CgOpts(6, 50, 0.0, 1, 0)
        r = krylov._CgResult()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = lib.pjds_cg_solve_static(ctypes.byref(D64.struct), ctypes.byref(Dlo.struct) if Dlo else None,
                                      bp.data_ptr(), x_st.data_ptr(), ctypes.byref(o), ctypes.byref(r),
                                      torch.cuda.current_stream().cuda_stream)
        assert rc == 0, pjds.lib().pjds_last_error()
        torch.cuda.synchronize()
        # nothing was allocated on the device by the second call (the first
        # may still load the module that holds the array, where the CUDA driver
        # loads modules lazily)
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        xs, xr = x_st.cpu().numpy(), x_ref.cpu().numpy()
        # tolerance of the CG tests: x within 1e-11 (relative, max norm), fp64 residual <= 1e-12
        assert np.max(np.abs(xs - xr)) <= 1e-11 * np.max(np.abs(xr)), call
        x = np.empty(A.n_rows)
        x[perm] = xs
        rel = np.linalg.norm(b - oracle_lib.crs_spmv(A, x)) / np.linalg.norm(b)
        assert rel <= 1e-12, (call, rel)
        assert r.outer == ref["outer"] and r.inner_total == ref["inner_total"]


def test_static_workspace_rejects_too_many_rows(mods):
    torch, pjds, krylov = mods
    A = synth.stencil27(g=51, seed=1)                  # 132651 rows > 131072
    D64, _ = _dev(pjds, A, "f64")
    v = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    with pytest.raises(pjds.PjdsError) as ei:
        krylov.cg_solve_static(D64, None, v, v.clone())
    assert ei.value.code == -1 and "131072" in str(ei.value)
