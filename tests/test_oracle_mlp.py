"""Pins for the fp64 cost-model oracle (oracle/mlp.py)."""
import numpy as np
import pytest


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 15))
    y = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] - X[:, 3]
    return X, y


def test_gradients_match_finite_differences():
    from oracle import mlp
    p = mlp.init(3)
    X, y = _data(40, 1)
    g = mlp.grads(p, X, y)
    rng = np.random.default_rng(5)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(p, X, y)
            flat[idx] = old - h
            lm = mlp.loss(p, X, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (k, idx)


def test_adam_first_step_closed_form():
    # at t = 1 the bias corrections make the step lr * g / (|g| + eps) = lr * sign(g)
    from oracle import mlp
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 0.0])}
    out = mlp.adam_step(dict(p), g, {}, 1, lr=0.01)
    assert np.allclose(out["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5], atol=1e-9)


def test_training_fits_a_linear_target():
    from oracle import mlp
    rng = np.random.default_rng(0)
    X = rng.standard_normal((256, 15))
    y = X @ rng.uniform(-1, 1, 15) + 0.3
    p, st = mlp.init(1), {}
    l0 = mlp.loss(p, X, y)
    for t in range(1, 1501):
        p = mlp.adam_step(p, mlp.grads(p, X, y), st, t, lr=3e-3)
    assert mlp.loss(p, X, y) < 1e-3 * l0


def test_planted_mistakes_are_caught():
    # a gradient that forgets the ReLU mask (or flips a sign) fails the
    # finite-difference pin
    from oracle import mlp
    p = mlp.init(4)
    X, y = _data(30, 2)
    g = mlp.grads(p, X, y)
    h = 1e-6
    flat = p["w1"].reshape(-1)
    old = flat[7]
    flat[7] = old + h
    lp = mlp.loss(p, X, y)
    flat[7] = old - h
    lm = mlp.loss(p, X, y)
    flat[7] = old
    fd = (lp - lm) / (2 * h)
    assert g["w1"].reshape(-1)[7] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    assert -g["w1"].reshape(-1)[7] != pytest.approx(fd, rel=1e-3) or fd == 0
    # unmasked backward through the first ReLU
    out, (Xc, z1, h1, z2, h2) = mlp.forward(p, X)
    d_out = 2.0 * (out - y) / len(y)
    d_h2 = np.outer(d_out, p["w3"]) * (z2 > 0)
    wrong = ((d_h2 @ p["w2"]).T @ X).reshape(-1)
    assert not np.allclose(wrong, g["w1"].reshape(-1), rtol=1e-6)
