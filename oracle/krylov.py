"""FP64 Krylov oracles (CG, Lanczos) — test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this.
Plain numpy in fp64 with the oracle's CRS product (oracle_crs_spmv) as the
matrix-vector step; no blocking, fusion or reordering of the textbook
recurrences. These are the references for the solver use the paper names as
the purpose of pJDS (Sect. 1.1: sparse eigenvalue and linear solvers; Sect. 2.1:
iterative methods run in the permuted basis; Sect. 4: a Lanczos-type
production eigensolver), where the GPU keeps values in fp32/bf16 and refines
in fp64.

Pins (tests/test_oracle_krylov.py): CG against numpy.linalg.solve and the
A-norm error decrease; Lanczos with k = n steps against numpy.linalg.eigvalsh
of the dense matrix, the three-term relation A V = V T + beta v e^T, and the
orthonormality of the basis for small k.
"""
from __future__ import annotations

import numpy as np

from . import crs_spmv


def cg(A, b: np.ndarray, iters: int, x0: np.ndarray | None = None):
    """Conjugate gradients (Hestenes-Stiefel), fp64, `iters` steps, no
    preconditioner. Returns (x, list of ||r_k||_2 with r_k the recursive
    residual, k = 0..iters)."""
    x = np.zeros(A.n_cols) if x0 is None else np.array(x0, np.float64)
    r = b - crs_spmv(A, x)
    p = r.copy()
    rr = float(r @ r)
    hist = [np.sqrt(rr)]
    for _ in range(iters):
        q = crs_spmv(A, p)
        pq = float(p @ q)
        if pq == 0.0:
            break
        alpha = rr / pq
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        hist.append(np.sqrt(rr))
    return x, hist


def lanczos(A, v0: np.ndarray, k: int, keep_basis: bool = False):
    """k steps of the symmetric Lanczos recurrence, fp64, no
    reorthogonalisation: beta_{j+1} v_{j+1} = A v_j - alpha_j v_j - beta_j v_{j-1}.
    Returns (alpha[k], beta[k+1] with beta[0] = 0, basis V (k x n) or None)."""
    n = A.n_rows
    v_prev = np.zeros(n)
    v = np.asarray(v0, np.float64) / np.linalg.norm(v0)
    alpha = np.zeros(k)
    beta = np.zeros(k + 1)
    V = np.zeros((k, n)) if keep_basis else None
    for j in range(k):
        if keep_basis:
            V[j] = v
        w = crs_spmv(A, v)
        alpha[j] = float(w @ v)
        w = w - alpha[j] * v - beta[j] * v_prev
        beta[j + 1] = float(np.linalg.norm(w))
        v_prev = v
        v = w / beta[j + 1] if beta[j + 1] != 0.0 else w
    return alpha, beta, V


def tridiag_eigvals(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Eigenvalues (ascending) of the Lanczos tridiagonal T_k (diagonal alpha,
    off-diagonal beta[1:k]) by numpy.linalg.eigvalsh."""
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[1:k], 1) + np.diag(beta[1:k], -1)
    return np.linalg.eigvalsh(T)


def ritz_pair(alpha, beta, V, which: str = "largest"):
    """Ritz value and Ritz vector y = V^T s of T_k's extreme eigenpair."""
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[1:k], 1) + np.diag(beta[1:k], -1)
    w, S = np.linalg.eigh(T)
    i = k - 1 if which == "largest" else 0
    return float(w[i]), V.T @ S[:, i]
