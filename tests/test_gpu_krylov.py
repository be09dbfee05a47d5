"""GPU Krylov drivers (pjds_cg_solve, pjds_lanczos, pjds_ritz_refine) against
the fp64 oracles. Solvers run in the permuted basis; results are mapped back
to the original basis with the permutation before every comparison.

Tolerances:
  CG (fp64 or refined mixed precision): the fp64 residual ||b - A x|| / ||b||,
    evaluated by the oracle's CRS product, <= 1e-12, and x within 1e-11
    (relative, max norm) of the oracle's fp64 CG solution (both are converged:
    the stencil matrices here have condition numbers near 25).
  Lanczos fp64: alpha_j, beta_j within 1e-10 (relative) of the oracle for the
    first 15 steps (rounding differences grow once orthogonality is lost),
    the extreme Ritz value within 1e-12.
  Lanczos fp32/bf16 values with fp32 vectors: extreme Ritz value within 1e-5
    (relative) of the fp64 oracle run on the same rounded values; the
    fp64-refined Rayleigh quotient within 1e-6 (fp32) / 5e-3 (bf16) of the
    fp64 oracle on the exact matrix, and its residual equal to the oracle's
    recomputation within 1e-6.
"""
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
    perm = H.perm.copy()
    return H.to_device("cuda"), perm


@pytest.fixture(scope="module")
def stencil():
    return synth.stencil27(g=20, p_drop=0.1, seed=7)


def _true_rel_residual(oracle_lib, A, x, b):
    return float(np.linalg.norm(b - oracle_lib.crs_spmv(A, x)) / np.linalg.norm(b))


@pytest.mark.parametrize("lo,max_outer,inner", [(None, 1, 300), ("f32", 6, 50), ("bf16", 20, 25)])
@pytest.mark.parametrize("graph", [True, False])
def test_cg_matches_fp64_oracle(mods, oracle_lib, stencil, lo, max_outer, inner, graph):
    torch, pjds, krylov = mods
    from oracle import krylov as ok
    A = stencil
    b = synth.vector(A.n_rows, seed=3)
    D64, perm = _dev(pjds, A, "f64")
    Dlo = _dev(pjds, A, lo)[0] if lo else None
    bp = torch.from_numpy(b[perm]).cuda()
    xp = torch.zeros_like(bp)
    res = krylov.cg_solve(D64, Dlo, bp, xp, max_outer=max_outer, inner_iters=inner, use_graph=graph)
    x = np.empty(A.n_rows)
    x[perm] = xp.cpu().numpy()
    rel = _true_rel_residual(oracle_lib, A, x, b)
    assert rel <= 1e-12, (rel, res)
    assert res["rel_residual"] == pytest.approx(rel, rel=1e-3, abs=1e-15)
    x_ref, _ = ok.cg(A, b, 300)
    assert np.max(np.abs(x - x_ref)) <= 1e-11 * np.max(np.abs(x_ref))
    h = res["history"]
    assert h[0] == pytest.approx(1.0) and h[-1] < 1e-12


def test_cg_is_deterministic_and_graph_equals_direct(mods, stencil):
    torch, pjds, krylov = mods
    A = stencil
    b = synth.vector(A.n_rows, seed=5)
    D64, perm = _dev(pjds, A, "f64")
    D32, _ = _dev(pjds, A, "f32")
    bp = torch.from_numpy(b[perm]).cuda()
    outs = []
    for graph in (True, True, False):
        xp = torch.zeros_like(bp)
        krylov.cg_solve(D64, D32, bp, xp, max_outer=3, inner_iters=20, use_graph=graph)
        outs.append(xp.cpu().numpy())
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
    assert np.array_equal(outs[0].view(np.uint64), outs[2].view(np.uint64))


def test_cg_rejects_bad_arguments(mods, stencil):
    torch, pjds, krylov = mods
    A = stencil
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64")  # not permuted
    D = H.to_device("cuda")
    v = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    with pytest.raises(pjds.PjdsError):
        krylov.cg_solve(D, None, v, v.clone())
    D32, _ = _dev(pjds, A, "f32")
    with pytest.raises(pjds.PjdsError):  # A_hi must be fp64
        krylov.cg_solve(D32, None, v, v.clone())


def test_lanczos_fp64_matches_oracle(mods, oracle_lib):
    torch, pjds, krylov = mods
    from oracle import krylov as ok
    A = synth.stencil27(g=16, seed=4)
    v0 = synth.vector(A.n_rows, seed=8)
    D, perm = _dev(pjds, A, "f64")
    k = 60
    alpha, beta, V = krylov.lanczos(D, torch.from_numpy(v0[perm]).cuda(), k, keep_basis=True)
    ra, rb, _ = ok.lanczos(A, v0, k)
    assert np.allclose(alpha[:15], ra[:15], rtol=1e-10, atol=0)
    assert np.allclose(beta[1:16], rb[1:16], rtol=1e-10, atol=0)
    assert beta[0] == 0.0
    th, _ = krylov.tridiag_extreme(alpha, beta)
    assert th == pytest.approx(ok.tridiag_eigvals(ra, rb)[-1], rel=1e-12)
    Vh = V.cpu().numpy()[:10]
    assert np.allclose(Vh @ Vh.T, np.eye(10), atol=1e-10)


def test_lanczos_graph_equals_direct(mods):
    torch, pjds, krylov = mods
    A = synth.stencil27(g=12, seed=4)
    D, perm = _dev(pjds, A, "f32")
    v0 = torch.from_numpy(synth.vector(A.n_rows, seed=2)[perm].astype(np.float32)).cuda()
    a1, b1, _ = krylov.lanczos(D, v0, 40, use_graph=True)
    a2, b2, _ = krylov.lanczos(D, v0, 40, use_graph=False)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_lanczos_low_precision_with_fp64_ritz_refinement(mods, oracle_lib, dtype):
    torch, pjds, krylov = mods
    from oracle import krylov as ok
    A = synth.stencil27(g=16, seed=4)
    v0 = synth.vector(A.n_rows, seed=8)
    Dlo, perm = _dev(pjds, A, dtype)
    D64, _ = _dev(pjds, A, "f64")
    k = 80
    alpha, beta, V = krylov.lanczos(Dlo, torch.from_numpy(v0[perm].astype(np.float32)).cuda(), k, keep_basis=True)
    ra, rb, RV = ok.lanczos(A, v0, k, keep_basis=True)
    th_ref, y_ref = ok.ritz_pair(ra, rb, RV)
    th, s = krylov.tridiag_extreme(alpha, beta)
    # the fp32 recurrence sees the dtype-rounded matrix: compare against the
    # oracle on the same rounded values for the unrefined Ritz value
    Ar = A._replace(val=oracle_lib.round_f32(A.val) if dtype == "f32" else oracle_lib.round_bf16(A.val))
    ra_r, rb_r, _ = ok.lanczos(Ar, v0, k)
    th_r = ok.tridiag_eigvals(ra_r, rb_r)[-1]
    assert th == pytest.approx(th_r, rel=1e-5)
    y, th_ref64, resid = krylov.ritz_refine(D64, V, s)
    # the Ritz vector approximates an eigenvector of the rounded matrix; its
    # fp64 Rayleigh quotient errs by about (rounding * ||A|| / gap)^2 * ||A||:
    # ~1e-10 relative for fp32 values, ~1e-3 for bf16 on this spectrum
    assert th_ref64 == pytest.approx(th_ref, rel=1e-6 if dtype == "f32" else 5e-3)
    yo = np.empty(A.n_rows)
    yo[perm] = y.cpu().numpy()
    r_or = np.linalg.norm(oracle_lib.crs_spmv(A, yo) - th_ref64 * yo) / np.linalg.norm(yo) / abs(th_ref64)
    assert resid == pytest.approx(r_or, rel=1e-6, abs=1e-14)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_lanczos_basis_rows_of_odd_length(mods, oracle_lib, dtype):
    # n = 17^3 = 4913: basis row j starts j * n elements in, so most rows are
    # not 16-byte aligned and take the element-wise stores; keeping the basis
    # changes no arithmetic, and the stored rows are the Lanczos vectors
    torch, pjds, krylov = mods
    from oracle import krylov as ok
    A = synth.stencil27(g=17, seed=5)
    assert A.n_rows % 2 == 1
    v0 = synth.vector(A.n_rows, seed=9)
    D, perm = _dev(pjds, A, dtype)
    v0t = torch.from_numpy(v0[perm]).to("cuda", D.vec_dtype)
    k = 30
    a1, b1, V = krylov.lanczos(D, v0t, k, keep_basis=True)
    a2, b2, _ = krylov.lanczos(D, v0t, k, keep_basis=False)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    Vh = V.double().cpu().numpy()
    v0n = v0t.double().cpu().numpy()
    assert np.allclose(Vh[0], v0n / np.linalg.norm(v0n), rtol=0, atol=1e-6 if dtype == "f32" else 1e-15)
    G = Vh[:8] @ Vh[:8].T
    assert np.allclose(G, np.eye(8), atol=1e-5 if dtype == "f32" else 1e-10)
    if dtype == "f64":
        ra, rb, _ = ok.lanczos(A, v0, k)
        assert np.allclose(a1[:10], ra[:10], rtol=1e-10, atol=0)
