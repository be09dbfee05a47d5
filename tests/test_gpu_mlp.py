"""Hand-written MLP kernels (training and inference) against the fp64 oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1112_5588_gb300 import build
    build.build()
    from paper_1112_5588_gb300 import learned
    return learned


def _to_oracle(m):
    return {"w1": np.array(m.w1, np.float64).reshape(64, 15), "b1": np.array(m.b1, np.float64),
            "w2": np.array(m.w2, np.float64).reshape(64, 64), "b2": np.array(m.b2, np.float64),
            "w3": np.array(m.w3, np.float64), "b3": np.array([m.b3], np.float64)}


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 15)).astype(np.float32)
    y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - X[:, 3]).astype(np.float32)
    return X, y


def test_forward_matches_oracle(L):
    from oracle import mlp as om
    m = L.init(2)
    m.b1[:] = np.linspace(-0.1, 0.1, 64)
    X, _ = _data(333, 1)  # ragged: not a multiple of the 64-sample tile
    got = L.predict(m, X)
    want, _ = om.forward(_to_oracle(m), X.astype(np.float64))
    assert np.allclose(got, want, rtol=1e-5, atol=1e-5)


def test_one_full_batch_adam_step_matches_oracle(L):
    from oracle import mlp as om
    m = L.init(3)
    X, y = _data(200, 4)
    p = _to_oracle(m)
    g = om.grads(p, X.astype(np.float64), y.astype(np.float64))
    p1 = om.adam_step({k: v.copy() for k, v in p.items()}, g, {}, 1, lr=1e-3)
    L.train(m, X, y, epochs=1, batch=10_000, lr=1e-3)
    q = _to_oracle(m)
    for k in p:
        # the first Adam step is lr * g / (|g| + eps): compare where |g| is not tiny
        big = np.abs(g[k]) > 1e-4 * np.abs(g[k]).max()
        assert np.allclose(q[k][big], p1[k][big], rtol=0, atol=2e-6), k


def test_full_batch_training_tracks_oracle_loss(L):
    from oracle import mlp as om
    m = L.init(4)
    X, y = _data(256, 5)
    p, st = _to_oracle(m), {}
    Xd, yd = X.astype(np.float64), y.astype(np.float64)
    ref = []
    for t in range(1, 41):
        p = om.adam_step(p, om.grads(p, Xd, yd), st, t, lr=2e-3)
        ref.append(om.loss(p, Xd, yd))
    hist = L.train(m, X, y, epochs=40, batch=256, lr=2e-3)
    assert np.allclose(hist, ref, rtol=2e-3)


def test_minibatch_training_fits_and_is_deterministic(L):
    X, y = _data(4000, 6)
    m1, m2 = L.init(7), L.init(7)
    L.fit_scaling(m1, X, y)
    L.fit_scaling(m2, X, y)
    h1 = L.train(m1, X, y, epochs=60, batch=512, lr=3e-3, seed=11)
    h2 = L.train(m2, X, y, epochs=60, batch=512, lr=3e-3, seed=11)
    assert h1[-1] < 0.05 * h1[0]
    assert np.array_equal(np.array(m1.w2), np.array(m2.w2))
    assert np.array_equal(h1, h2)
