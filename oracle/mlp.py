"""FP64 oracle of the learned SO(3) proposal network (test infrastructure only).

Network (the proposal of the 3D matching workload): x = the real channels of
the component correlations at a voxel divided by their L2 norm,
    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  o = W3 h2 + b3,
    q^ = o / |o|   (a unit quaternion),
loss l = mean(1 - <q^, q*>^2)  (invariant under q* -> -q*, which encode the
same rotation).  Gradients are derived by hand below; the finite-difference
test pins them.
"""
from __future__ import annotations

import numpy as np


def forward(p, X):
    X = np.asarray(X, np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    o = h2 @ p["W3"].T + p["b3"]
    return dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, o=o)


def quaternion(o):
    return o / np.linalg.norm(o, axis=1, keepdims=True)


def loss(o, qt):
    q = quaternion(o)
    d = np.sum(q * qt, axis=1)
    return float(np.mean(1.0 - d * d))


def backward(p, cache, qt):
    """Gradients of the mean loss w.r.t. every parameter."""
    o = cache["o"]
    n = o.shape[0]
    norm = np.linalg.norm(o, axis=1, keepdims=True)
    q = o / norm
    d = np.sum(q * qt, axis=1, keepdims=True)
    dq = -2.0 * d * qt / n                      # d loss / d q^
    do = (dq - q * np.sum(dq * q, axis=1, keepdims=True)) / norm   # through q = o / |o|
    g = {}
    g["W3"] = do.T @ cache["h2"]
    g["b3"] = do.sum(axis=0)
    dh2 = do @ p["W3"]
    dz2 = dh2 * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = dz1.T @ cache["X"]
    g["b1"] = dz1.sum(axis=0)
    return g


def init_params(rng, n_in, hidden=256):
    """He-initialised weights, zero biases (FP64)."""
    def he(o, i):
        return rng.standard_normal((o, i)) * np.sqrt(2.0 / i)
    return dict(W1=he(hidden, n_in), b1=np.zeros(hidden), W2=he(hidden, hidden), b2=np.zeros(hidden),
                W3=he(4, hidden) * 0.5, b3=np.zeros(4))


def adam_step(p, g, state, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of every parameter;
    state holds the moments m, v and the step count t (start: {})."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = {}
    for k, w in p.items():
        m = b1 * state.get("m_" + k, np.zeros_like(w)) + (1 - b1) * g[k]
        v = b2 * state.get("v_" + k, np.zeros_like(w)) + (1 - b2) * g[k] ** 2
        state["m_" + k], state["v_" + k] = m, v
        mhat = m / (1 - b1 ** t)
        vhat = v / (1 - b2 ** t)
        out[k] = w - lr * mhat / (np.sqrt(vhat) + eps)
    return out
