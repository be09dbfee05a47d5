"""Write bounds of every GPU entry point, checked with canaries.

Each output (and each caller workspace) is a view into the middle of a
larger buffer whose head and tail hold a fixed bit pattern; after the call
the pattern must be intact on both sides, so a write past either end of an
output is caught on the host. The matrices are ragged (row counts that are
not multiples of the block size, empty rows) so that tails and padding
rows are exercised.
"""
import ctypes

import numpy as np
import pytest

import synth
from synth import tiny

pytestmark = pytest.mark.gpu

G = 4096          # canary elements on each side (a multiple of 64: views stay 512-byte aligned)
PATTERN = 0x5A    # canary byte


@pytest.fixture(scope="module")
def mods():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import batch, krylov, pjds
    return torch, pjds, batch, krylov


def guarded(torch, n, dtype, device="cuda", pin=False):
    """(buffer, view of n elements in its middle); canary bytes elsewhere."""
    esz = torch.empty(0, dtype=dtype).element_size()
    raw = torch.full(((n + 2 * G) * esz,), PATTERN, dtype=torch.uint8)
    raw = raw.pin_memory() if pin else raw.to(device)
    buf = raw.view(dtype)
    return raw, buf[G:G + n]


def intact(torch, raw, n, dtype):
    esz = torch.empty(0, dtype=dtype).element_size()
    r = raw.cpu().numpy()
    return bool((r[:G * esz] == PATTERN).all() and (r[(G + n) * esz:] == PATTERN).all())


MATS = [lambda: tiny.random_lengths(1037, 1037, max_len=90, seed=81, p_empty=0.2),
        lambda: synth.zipf_rows(5_003, s=1.8, len_max=400, seed=82),
        lambda: synth.hmep_like(n=20_011, seed=83)]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("permute", [False, True])
def test_spmv_and_ellr_write_only_y(mods, dtype, permute):
    torch, pjds, batch, krylov = mods
    for make in MATS:
        A = make()
        for b in (32, 256):
            D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=b, dtype=dtype,
                                 permute_cols=permute).to_device("cuda")
            x = torch.rand(A.n_cols, device="cuda", dtype=D.vec_dtype)
            for cfg in (dict(), dict(threads_per_row=1), dict(threads_per_row=8, block_threads=64),
                        dict(rows_per_thread=2), dict(rows_per_thread=4), dict(staged=1), dict(tile_order=1),
                        dict(rows_per_thread=2, tile_order=1), dict(threads_per_row=4, tile_order=1),
                        dict(plan=1), dict(plan=1, index64=1)):
                raw, y = guarded(torch, A.n_rows, D.vec_dtype)
                pjds.pjds_spmv_cfg(D, x, y, **cfg)
                torch.cuda.synchronize()
                assert intact(torch, raw, A.n_rows, D.vec_dtype), (cfg, b, A.n_rows)
                assert torch.isfinite(y.float()).all(), cfg
            # the pattern product (one thread per row in both tile orders, T threads per row, the plan)
            for cfg in (dict(threads_per_row=1), dict(threads_per_row=1, tile_order=1), dict(threads_per_row=4),
                        dict(plan=1)):
                raw, y = guarded(torch, A.n_rows, D.vec_dtype)
                pjds.pjds_spmv_pattern(D, x, y, **cfg)
                torch.cuda.synchronize()
                assert intact(torch, raw, A.n_rows, D.vec_dtype), ("pattern", cfg, b, A.n_rows)
                assert torch.isfinite(y.float()).all(), cfg
        E = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype=dtype).to_device("cuda")
        raw, y = guarded(torch, A.n_rows, E.vec_dtype)
        pjds.ellr_spmv(E, torch.rand(A.n_cols, device="cuda", dtype=E.vec_dtype), y)
        torch.cuda.synchronize()
        assert intact(torch, raw, A.n_rows, E.vec_dtype)


def test_permute_spmm_batch_write_only_their_outputs(mods):
    torch, pjds, batch, krylov = mods
    A = MATS[0]()
    D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, permute_cols=True).to_device("cuda")
    v = torch.rand(A.n_rows, device="cuda", dtype=torch.float64)
    for fn in (pjds.pjds_permute, pjds.pjds_unpermute):
        raw, out = guarded(torch, A.n_rows, torch.float64)
        fn(D, v, out)
        torch.cuda.synchronize()
        assert intact(torch, raw, A.n_rows, torch.float64)
    for dtype, k in (("f64", 2), ("f64", 16), ("f32", 4), ("f32", 32), ("bf16", 8)):
        Dk = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype).to_device("cuda")
        X = torch.rand(A.n_cols, k, device="cuda", dtype=Dk.vec_dtype)
        raw, flat = guarded(torch, A.n_rows * k, Dk.vec_dtype)
        batch.spmm(Dk, X, flat.view(A.n_rows, k))
        torch.cuda.synchronize()
        assert intact(torch, raw, A.n_rows * k, Dk.vec_dtype), (dtype, k)
        raw, flat = guarded(torch, A.n_rows * k, Dk.vec_dtype)
        batch.spmm_pattern(Dk, X, flat.view(A.n_rows, k))
        torch.cuda.synchronize()
        assert intact(torch, raw, A.n_rows * k, Dk.vec_dtype), ("pattern", dtype, k)
    mats = [m() for m in MATS]
    devs = [pjds.pjds_create(M.n_rows, M.n_cols, M.row_ptr, M.col, M.val, b=32).to_device("cuda") for M in mats]
    xs = [torch.rand(M.n_cols, device="cuda", dtype=torch.float64) for M in mats]
    for kw in (dict(), dict(rule=(4, 16, 64)), dict(lanes=[8, 2, 1])):
        guards = [guarded(torch, M.n_rows, torch.float64) for M in mats]
        B = batch.Batch(devs, xs, [g[1] for g in guards], **kw)
        B.run(use_graph=True)
        torch.cuda.synchronize()
        assert all(intact(torch, raw, M.n_rows, torch.float64) for (raw, _), M in zip(guards, mats)), kw
        B.run_pattern()
        torch.cuda.synchronize()
        assert all(intact(torch, raw, M.n_rows, torch.float64) for (raw, _), M in zip(guards, mats)), kw
        B.destroy()


def test_krylov_workspaces_and_outputs_stay_in_bounds(mods):
    torch, pjds, batch, krylov = mods
    S = synth.stencil27(g=13, seed=84)  # 2197 rows (odd)
    D64 = pjds.pjds_create(S.n_rows, S.n_cols, S.row_ptr, S.col, S.val, dtype="f64",
                           permute_cols=True).to_device("cuda")
    D32 = pjds.pjds_create(S.n_rows, S.n_cols, S.row_ptr, S.col, S.val, dtype="f32",
                           permute_cols=True).to_device("cuda")
    b = torch.rand(S.n_rows, device="cuda", dtype=torch.float64)
    for lo, vec in ((None, 0), (D32, 1)):
        need = krylov.cg_workspace_bytes(S.n_rows, D64.n_pad, vec)
        wraw, work = guarded(torch, need, torch.uint8)
        xraw, x = guarded(torch, S.n_rows, torch.float64)
        x.zero_()
        krylov.cg_solve(D64, lo, b, x, max_outer=2, inner_iters=10, work=work)
        torch.cuda.synchronize()
        assert intact(torch, wraw, need, torch.uint8) and intact(torch, xraw, S.n_rows, torch.float64)
    steps = 12
    for D in (D64, D32):
        need = ctypes.c_size_t()
        vec = 0 if D is D64 else 1
        assert krylov._lib.pjds_lanczos_workspace_bytes(S.n_rows, D.n_pad, vec, steps, ctypes.byref(need)) == 0
        wraw, work = guarded(torch, need.value, torch.uint8)
        braw, basis = guarded(torch, steps * S.n_rows, D.vec_dtype)
        v0 = torch.rand(S.n_rows, device="cuda", dtype=D.vec_dtype)
        al, be = np.zeros(steps), np.zeros(steps + 1)
        rc = krylov._lib.pjds_lanczos(ctypes.byref(D.struct), v0.data_ptr(), steps, al.ctypes.data, be.ctypes.data,
                                      basis.data_ptr(), 1, work.data_ptr(), need.value,
                                      torch.cuda.current_stream().cuda_stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert intact(torch, wraw, need.value, torch.uint8)
        assert intact(torch, braw, steps * S.n_rows, D.vec_dtype)


def test_host_stream_writes_only_its_host_outputs(mods):
    torch, pjds, batch, krylov = mods
    A = MATS[2]()
    D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32).to_device("cuda")
    xs = [torch.rand(A.n_cols, dtype=torch.float64).pin_memory() for _ in range(3)]
    guards = [guarded(torch, A.n_rows, torch.float64, pin=True) for _ in range(3)]
    dx = [guarded(torch, A.n_cols, torch.float64) for _ in range(2)]
    dy = [guarded(torch, A.n_rows, torch.float64) for _ in range(2)]
    pjds.pjds_spmv_host_stream(D, xs, [g[1] for g in guards], [g[1] for g in dx], [g[1] for g in dy])
    assert all(intact(torch, raw, A.n_rows, torch.float64) for raw, _ in guards)
    assert all(intact(torch, raw, A.n_cols, torch.float64) for raw, _ in dx)
    assert all(intact(torch, raw, A.n_rows, torch.float64) for raw, _ in dy)
