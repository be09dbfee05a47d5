"""Pins for the fp64 CG and Lanczos oracles (oracle/krylov.py)."""
import numpy as np
import pytest

import synth
from synth import tiny


def _spd_dense(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.uniform(-1, 1, (n, n)) * (rng.random((n, n)) < 0.2)
    S = M + M.T
    np.fill_diagonal(S, 0.0)
    np.fill_diagonal(S, np.abs(S).sum(1) + 1.0)
    return S


def test_cg_matches_dense_solve():
    from oracle import krylov
    D = _spd_dense(80, 1)
    A = tiny.from_dense(D)
    b = np.random.default_rng(2).uniform(-1, 1, 80)
    x, hist = krylov.cg(A, b, 200)
    assert np.allclose(x, np.linalg.solve(D, b), rtol=0, atol=1e-12)
    assert hist[-1] < 1e-12 * hist[0]


def test_cg_a_norm_error_decreases():
    # CG minimises the A-norm of the error over growing Krylov spaces
    from oracle import krylov
    D = _spd_dense(60, 3)
    A = tiny.from_dense(D)
    b = np.random.default_rng(4).uniform(-1, 1, 60)
    xs = np.linalg.solve(D, b)
    errs = []
    for k in range(0, 25, 3):
        x, _ = krylov.cg(A, b, k)
        e = x - xs
        errs.append(float(e @ D @ e))
    assert all(e2 <= e1 * (1 + 1e-9) for e1, e2 in zip(errs, errs[1:]))


def test_pins_catch_planted_mistakes(monkeypatch):
    # plant a dropped term in the oracle's matrix-vector step: both the CG and
    # the Lanczos pins must fail
    import oracle
    from oracle import krylov
    D = _spd_dense(50, 5)
    A = tiny.from_dense(D)
    b = np.random.default_rng(1).uniform(-1, 1, 50)
    good = oracle.crs_spmv

    def dropped(M, v):
        y = good(M, v)
        for i in range(M.n_rows):
            k = M.row_ptr[i + 1] - 1
            if k >= M.row_ptr[i]:
                y[i] -= M.val[k] * v[M.col[k]]
        return y
    monkeypatch.setattr(krylov, "crs_spmv", dropped)
    x, _ = krylov.cg(A, b, 200)
    assert not np.allclose(x, np.linalg.solve(D, b), rtol=0, atol=1e-12)
    alpha, beta, _ = krylov.lanczos(A, np.ones(50), 50)
    assert abs(krylov.tridiag_eigvals(alpha, beta)[-1] - np.linalg.eigvalsh(D)[-1]) > 1e-6


def test_lanczos_full_steps_give_spectrum():
    from oracle import krylov
    D = _spd_dense(40, 6)
    A = tiny.from_dense(D)
    v0 = np.random.default_rng(7).uniform(-1, 1, 40)
    alpha, beta, V = krylov.lanczos(A, v0, 40, keep_basis=True)
    ev = np.linalg.eigvalsh(D)
    th = krylov.tridiag_eigvals(alpha, beta)
    assert abs(th[-1] - ev[-1]) < 1e-9 * ev[-1]
    assert abs(th[0] - ev[0]) < 1e-9 * ev[-1]


def test_lanczos_three_term_relation_and_orthonormality():
    from oracle import krylov
    A = synth.stencil27(g=10, seed=3)
    D = np.zeros((A.n_rows, A.n_rows))
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    D[rows, A.col] = A.val
    k = 12
    v0 = synth.vector(A.n_rows, seed=9)
    alpha, beta, V = krylov.lanczos(A, v0, k, keep_basis=True)
    T = np.diag(alpha) + np.diag(beta[1:k], 1) + np.diag(beta[1:k], -1)
    # A V^T = V^T T + beta_k v_k e_k^T (columns of V^T are the Lanczos vectors)
    R = D @ V.T - V.T @ T
    assert np.allclose(R[:, :-1], 0, atol=1e-12)
    assert np.allclose(V @ V.T, np.eye(k), atol=1e-10)


def test_ritz_pair_is_accurate_for_extreme_eigenvalue():
    from oracle import krylov
    D = _spd_dense(120, 8)
    A = tiny.from_dense(D)
    v0 = np.random.default_rng(1).uniform(-1, 1, 120)
    alpha, beta, V = krylov.lanczos(A, v0, 60, keep_basis=True)
    th, y = krylov.ritz_pair(alpha, beta, V)
    assert np.linalg.norm(D @ y - th * y) < 1e-8 * th
    assert th == pytest.approx(np.linalg.eigvalsh(D)[-1], rel=1e-12)
