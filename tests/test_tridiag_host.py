"""Host-side tridiagonal eigenpair (pjds_tridiag_extreme) against numpy.linalg.eigh."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def K():
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import krylov
    return krylov


def _T(a, b):
    k = len(a)
    return np.diag(a) + np.diag(b[1:k], 1) + np.diag(b[1:k], -1)


@pytest.mark.parametrize("k", [1, 2, 3, 10, 57, 200])
@pytest.mark.parametrize("seed", range(3))
def test_extreme_eigenpairs(K, k, seed):
    rng = np.random.default_rng(seed * 100 + k)
    a = rng.uniform(-5, 20, k)
    b = np.concatenate([[0.0], rng.uniform(0.01, 3, k)])
    w, V = np.linalg.eigh(_T(a, b))
    for which, idx in (("largest", -1), ("smallest", 0)):
        th, s = K.tridiag_extreme(a, b, which)
        assert th == pytest.approx(w[idx], abs=1e-12 * max(1.0, abs(w).max()))
        assert np.linalg.norm(_T(a, b) @ s - th * s) < 1e-10 * max(1.0, abs(w).max())
        assert abs(np.linalg.norm(s) - 1) < 1e-12


def test_lanczos_like_clustered_spectrum(K):
    # a tridiagonal from the fp64 Lanczos oracle on a stencil: converged
    # extreme Ritz values come in near-copies (loss of orthogonality)
    import synth
    from oracle import krylov as ok
    A = synth.stencil27(g=14, seed=2)
    alpha, beta, _ = ok.lanczos(A, synth.vector(A.n_rows, seed=1), 150)
    w = np.linalg.eigvalsh(_T(alpha, beta))
    th, s = K.tridiag_extreme(alpha, beta, "largest")
    assert th == pytest.approx(w[-1], rel=1e-13)
    assert np.linalg.norm(_T(alpha, beta) @ s - th * s) < 1e-9 * w[-1]


def test_bad_arguments(K):
    from paper_1112_5588_gb300.pjds import PjdsError
    with pytest.raises(PjdsError):
        K.tridiag_extreme(np.zeros(0), np.zeros(1))
