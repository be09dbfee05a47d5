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


@pytest.mark.parametrize("lo,max_outer,inner", [("f32", 6, 50), ("bf16", 12, 25)])
def test_stencil_cg_refined_full(P, oracle_lib, stencil, lo, max_outer, inner):
    # the 300-step refined CG of the precision workload at full size: the fp64
    # residual of the returned solution, evaluated by the oracle, is <= 1e-12
    import torch
    from paper_1112_5588_gb300 import krylov
    A = stencil
    H64 = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64", permute_cols=True)
    perm = H64.perm.copy()
    D64 = H64.to_device("cuda")
    H64.destroy()
    Dlo = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=lo, permute_cols=True).to_device("cuda")
    b = synth.vector(A.n_rows, seed=1235)
    bp = torch.from_numpy(b[perm]).cuda()
    xp = torch.zeros_like(bp)
    res = krylov.cg_solve(D64, Dlo, bp, xp, max_outer=max_outer, inner_iters=inner)
    x = np.empty(A.n_rows)
    x[perm] = xp.cpu().numpy()
    rel = np.linalg.norm(b - oracle_lib.crs_spmv(A, x)) / np.linalg.norm(b)
    assert rel <= 1e-12, (rel, res)
    assert res["inner_total"] == 300


def test_dlr_spmm_k32_full(P, oracle_lib):
    # block product of the batching workload at full size: DLR-like N = 280k,
    # 144 nonzeros per row, fp32, k = 32
    import torch
    from paper_1112_5588_gb300 import batch
    A = synth.block_dense(n_brow=70_000, bs=4, nb=36, frac=0.05, seed=1234)
    k = 32
    X = np.random.default_rng(3).uniform(-1, 1, (A.n_cols, k)).astype(np.float32)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f32")
    D = H.to_device("cuda")
    Xt = torch.from_numpy(X).cuda()
    Yt = torch.empty(A.n_rows, k, device="cuda")
    batch.spmm(D, Xt, Yt)
    torch.cuda.synchronize()
    Ar = A._replace(val=oracle_lib.round_f32(A.val))
    Xd = X.astype(np.float64)
    Yr = oracle_lib.crs_spmm(Ar, Xd)
    S = oracle_lib.crs_spmm(Ar._replace(val=np.abs(Ar.val)), np.abs(Xd))
    Y = Yt.double().cpu().numpy()
    lens = np.diff(A.row_ptr)
    for c in range(k):
        r = parity.check_fp32(Y[:, c], Yr[:, c], S[:, c], lens)
        assert r["ok"], (c, r)


def test_batch_64_uneven_full(P, oracle_lib):
    # the 64-matrix batch of the batching workload (N log-uniform in [10k, 500k],
    # Zipf(2) rows capped at 512, fp64), one persistent graph launch
    import torch
    from paper_1112_5588_gb300 import batch
    rng = np.random.default_rng(1234)
    sizes = np.exp(rng.uniform(np.log(10_000), np.log(500_000), 64)).astype(int)
    mats, devs, xs, ys = [], [], [], []
    for m, n in enumerate(sizes):
        M = synth.zipf_rows(int(n), s=2.0, len_max=512, seed=1234 + m)
        devs.append(P.pjds_create(M.n_rows, M.n_cols, M.row_ptr, M.col, M.val, b=32).to_device("cuda"))
        xs.append(torch.from_numpy(synth.vector(M.n_cols, seed=m)).cuda())
        ys.append(torch.full((M.n_rows,), float("nan"), dtype=torch.float64, device="cuda"))
        mats.append(M)
    B = batch.Batch(devs, xs, ys)
    B.run(use_graph=True)
    torch.cuda.synchronize()
    for M, x, y in zip(mats, xs, ys):
        xh = x.cpu().numpy()
        r = parity.check_fp64(y.cpu().numpy(), oracle_lib.crs_spmv(M, xh), oracle_lib.crs_absmv(M, xh),
                              np.diff(M.row_ptr))
        assert r["ok"], r
    B.destroy()


def test_stencil_lanczos_f32_ritz_refined_full(P, oracle_lib, stencil):
    # the 200-step Lanczos of the precision workload at full size: fp32 values
    # and vectors, the extreme Ritz pair refined in fp64; the refined Rayleigh
    # quotient and residual equal the oracle's recomputation from the returned
    # vector, and the refined value agrees with a 200-step fp64 run
    import torch
    from paper_1112_5588_gb300 import krylov
    A = stencil
    H32 = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f32", permute_cols=True)
    perm = H32.perm.copy()
    D32 = H32.to_device("cuda")
    H32.destroy()
    D64 = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64",
                        permute_cols=True).to_device("cuda")
    v0 = synth.vector(A.n_rows, seed=1236)[perm]
    thetas = {}
    for D in (D32, D64):
        alpha, beta, V = krylov.lanczos(D, torch.from_numpy(v0).to("cuda", D.vec_dtype), 200, keep_basis=True)
        th, s = krylov.tridiag_extreme(alpha, beta)
        yv, th_ref, resid = krylov.ritz_refine(D64, V, s)
        y = np.empty(A.n_rows)
        y[perm] = yv.cpu().numpy()
        Ay = oracle_lib.crs_spmv(A, y)
        rq = float(y @ Ay / (y @ y))
        assert th_ref == pytest.approx(rq, rel=1e-13)
        assert resid == pytest.approx(float(np.linalg.norm(Ay - rq * y) / np.linalg.norm(y) / abs(rq)), rel=1e-6)
        thetas[D.dtype] = th_ref
        del V
        torch.cuda.empty_cache()
    assert thetas[1] == pytest.approx(thetas[0], rel=1e-10)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_dlr_default_paired_rows_full(P, oracle_lib, dtype):
    # the single product on the DLR-like matrix (280k rows of 144, 4x4 blocks):
    # the default pairs rows (pair_share 1000); every element within the fp32
    # bound of the oracle and bit for bit the one-row-per-thread product
    import torch
    A = synth.block_dense(n_brow=70_000, bs=4, nb=36, frac=0.05, seed=1234)
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype)
    assert H.pair_share == 1000
    D = H.to_device("cuda")
    H.destroy()
    assert P.pjds_spmv_resolve(D)["rows_per_thread"] == 2
    x = synth.vector(A.n_cols, seed=31).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    y = torch.full((A.n_rows,), float("nan"), device="cuda")
    P.pjds_spmv(D, xt, y)
    y1 = torch.full((A.n_rows,), float("nan"), device="cuda")
    P.pjds_spmv_cfg(D, xt, y1, rows_per_thread=1, threads_per_row=1)
    torch.cuda.synchronize()
    assert torch.equal(y, y1)
    Ar = A._replace(val=oracle_lib.round_f32(A.val) if dtype == "f32" else oracle_lib.round_bf16(A.val))
    xd = x.astype(np.float64)
    r = parity.check_fp32(y.double().cpu().numpy(), oracle_lib.crs_spmv(Ar, xd), oracle_lib.crs_absmv(Ar, xd),
                          np.diff(A.row_ptr))
    assert r["ok"], r


def _partly_shared_dlr():
    """The DLR-like matrix with entry 7 of every fifth row dropped: rows of 143
    sort behind those of 144, so about half the pairs of sorted rows no longer
    share their columns and some pairs hold rows of both lengths."""
    A = synth.block_dense(n_brow=70_000, bs=4, nb=36, frac=0.05, seed=1234)
    drop = np.arange(A.n_rows) % 5 == 1
    keep = np.ones(len(A.col), bool)
    keep[A.row_ptr[:-1][drop] + 7] = False
    rp = np.zeros(A.n_rows + 1, np.int64)
    np.cumsum(np.diff(A.row_ptr) - drop, out=rp[1:])
    return A._replace(row_ptr=rp, col=A.col[keep], val=A.val[keep])


def _odd_dlr():
    """The DLR-like matrix with one more row (a single entry): an odd row count,
    so the last pair of sorted rows holds one row."""
    A = synth.block_dense(n_brow=70_000, bs=4, nb=36, frac=0.05, seed=1234)
    return A._replace(n_rows=A.n_rows + 1, row_ptr=np.append(A.row_ptr, A.row_ptr[-1] + 1),
                      col=np.append(A.col, np.int32(5)), val=np.append(A.val, 0.75))


@pytest.mark.parametrize("which,dtype,k", [("dlr", "f32", 8), ("dlr", "f32", 64), ("dlr", "bf16", 16),
                                           ("dlr", "bf16", 32), ("partly", "f32", 8), ("partly", "bf16", 32),
                                           ("odd", "bf16", 16)])
def test_spmm_paired_rows_full(P, oracle_lib, which, dtype, k):
    # the block product with one thread per pair of rows (block-structured
    # matrices, fp32 / bf16, k a multiple of 8): every element within the fp32
    # bound, columns bit for bit the single product with one row per thread,
    # and its pattern product (the gather ceiling) against the oracle's
    import torch
    from paper_1112_5588_gb300 import batch
    A = {"dlr": lambda: synth.block_dense(n_brow=70_000, bs=4, nb=36, frac=0.05, seed=1234),
         "partly": _partly_shared_dlr, "odd": _odd_dlr}[which]()
    H = P.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dtype)
    assert H.pair_share >= 500, H.pair_share
    D = H.to_device("cuda")
    H.destroy()
    X = np.random.default_rng(k).uniform(-1, 1, (A.n_cols, k)).astype(np.float32)
    Xt = torch.from_numpy(X).cuda()
    Yt = torch.full((A.n_rows, k), float("nan"), device="cuda")
    batch.spmm(D, Xt, Yt)
    torch.cuda.synchronize()
    Ar = A._replace(val=oracle_lib.round_f32(A.val) if dtype == "f32" else oracle_lib.round_bf16(A.val))
    Xd = X.astype(np.float64)
    Yr = oracle_lib.crs_spmm(Ar, Xd)
    S = oracle_lib.crs_spmm(Ar._replace(val=np.abs(Ar.val)), np.abs(Xd))
    Y = Yt.double().cpu().numpy()
    lens = np.diff(A.row_ptr)
    for c in range(k):
        r = parity.check_fp32(Y[:, c], Yr[:, c], S[:, c], lens)
        assert r["ok"], (c, r)
    for c in (0, k - 1):
        y1 = torch.empty(A.n_rows, device="cuda")
        P.pjds_spmv_cfg(D, Xt[:, c].contiguous(), y1, threads_per_row=1, rows_per_thread=1)
        torch.cuda.synchronize()
        assert torch.equal(y1, Yt[:, c].contiguous()), c
    batch.spmm_pattern(D, Xt, Yt)
    torch.cuda.synchronize()
    ones = A._replace(val=np.ones_like(A.val))
    Yp = oracle_lib.crs_spmm(ones, Xd)
    Sp = oracle_lib.crs_spmm(ones, np.abs(Xd))
    Y = Yt.double().cpu().numpy()
    for c in (0, k // 2, k - 1):
        assert parity.check_fp32(Y[:, c], Yp[:, c], Sp[:, c], lens)["ok"], c
