"""Plain FP64 CPU reference of the corner-guidance MLP (TEST INFRASTRUCTURE).

The network the CUDA path trains: 18 per-column features -> 64 -> 64 -> 1,
ReLU after the two hidden layers, a sigmoid output read as the probability
that the column ends at a bound after the corner phase, and the mean binary
cross-entropy as the loss.  Weights are W1 (64 x 18), b1 (64), W2 (64 x 64),
b2 (64), w3 (64), b3 (scalar).  Written as whole-matrix numpy operations in
the order of the chain rule; pinned by central finite differences in the
tests.  Shares no code with the CUDA kernels.
"""
from __future__ import annotations

import numpy as np

IN, HID = 18, 64


def init_weights(seed: int = 0):
    """He-normal hidden layers, small output layer (a reading; any init works)."""
    rng = np.random.default_rng(seed)
    return dict(
        W1=rng.standard_normal((HID, IN)) * np.sqrt(2.0 / IN),
        b1=np.zeros(HID),
        W2=rng.standard_normal((HID, HID)) * np.sqrt(2.0 / HID),
        b2=np.zeros(HID),
        w3=rng.standard_normal(HID) * np.sqrt(1.0 / HID),
        b3=np.zeros(()),
    )


def forward(w, X):
    """Returns (p, cache): p = sigmoid(w3 . relu(W2 relu(W1 x + b1) + b2) + b3)."""
    Z1 = X @ w["W1"].T + w["b1"]
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ w["W2"].T + w["b2"]
    A2 = np.maximum(Z2, 0.0)
    o = A2 @ w["w3"] + w["b3"]
    p = 1.0 / (1.0 + np.exp(-o))
    return p, dict(X=X, Z1=Z1, A1=A1, Z2=Z2, A2=A2, o=o)


def bce(p, y):
    """Mean binary cross-entropy, clipped away from log(0)."""
    q = np.clip(p, 1e-12, 1 - 1e-12)
    return float(-np.mean(y * np.log(q) + (1 - y) * np.log(1 - q)))


def loss_of(w, X, y):
    return bce(forward(w, X)[0], y)


def gradients(w, X, y):
    """d(mean BCE)/d(weights) by the chain rule: d o = (p - y) / N."""
    p, c = forward(w, X)
    N = X.shape[0]
    do = (p - y) / N
    g = dict(w3=c["A2"].T @ do, b3=np.asarray(do.sum()))
    dA2 = np.outer(do, w["w3"])
    dZ2 = dA2 * (c["Z2"] > 0)
    g["W2"] = dZ2.T @ c["A1"]
    g["b2"] = dZ2.sum(axis=0)
    dA1 = dZ2 @ w["W2"]
    dZ1 = dA1 * (c["Z1"] > 0)
    g["W1"] = dZ1.T @ c["X"]
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam_step(w, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Kingma & Ba (2015) Adam with bias correction; state holds m, v, t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in w:
        m = state.setdefault("m_" + k, np.zeros_like(w[k]))
        v = state.setdefault("v_" + k, np.zeros_like(w[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        w[k] = w[k] - lr * mh / (np.sqrt(vh) + eps)
    return w
