"""FP64 reference of the learned tuner's cost model — test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this.
A two-hidden-layer perceptron with ReLU, written as plain numpy matrix
products in the textbook order, its mean-squared-error loss, the gradients by
the chain rule, and one Adam step (Kingma & Ba, "Adam: A Method for Stochastic
Optimization", ICLR 2015, Algorithm 1). The model predicts the (standardised)
logarithm of a kernel's time from standardised matrix features and a launch
candidate; the tuner picks the candidate with the smallest prediction.

Pins (tests/test_oracle_mlp.py): gradients against central finite
differences, the Adam step against its closed form on a hand-made case, a
linear target that training must fit, and planted mistakes.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 15, 64  # inputs: 8 matrix features + the 7-entry candidate encoding


def init(seed: int = 0):
    """He-uniform weights, zero biases (dict of fp64 arrays)."""
    rng = np.random.default_rng(seed)

    def he(fan_out, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, (fan_out, fan_in))
    return {"w1": he(N_H, N_IN), "b1": np.zeros(N_H), "w2": he(N_H, N_H), "b2": np.zeros(N_H),
            "w3": he(1, N_H)[0], "b3": np.zeros(1)}


def forward(p, X):
    """(prediction [n], cache) for inputs X [n, N_IN]."""
    z1 = X @ p["w1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["w2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["w3"] + p["b3"][0]
    return out, (X, z1, h1, z2, h2)


def loss(p, X, y) -> float:
    out, _ = forward(p, X)
    return float(np.mean((out - y) ** 2))


def grads(p, X, y):
    """Gradients of the mean squared error with respect to every parameter."""
    n = X.shape[0]
    out, (X, z1, h1, z2, h2) = forward(p, X)
    d_out = 2.0 * (out - y) / n
    g = {"w3": h2.T @ d_out, "b3": np.array([d_out.sum()])}
    d_h2 = np.outer(d_out, p["w3"]) * (z2 > 0)
    g["w2"] = d_h2.T @ h1
    g["b2"] = d_h2.sum(0)
    d_h1 = (d_h2 @ p["w2"]) * (z1 > 0)
    g["w1"] = d_h1.T @ X
    g["b1"] = d_h1.sum(0)
    return g


def adam_step(p, g, state, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step count t >= 1) of every parameter, in place."""
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
