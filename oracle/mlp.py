"""FP64 reference of the learned warm start's network (TEST INFRASTRUCTURE ONLY).

The network maps the 12 contact features (their definitions are in the
header of ``ovl_oracle.c``) to the three impulses of the contact divided by
its scale s: y = x[4:7] + W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3, with
layers 12-64-64-3.  Features 4-6 are the previous-step impulses / s, so the
layers learn a correction to the method's own warm start (zero for a new
contact's missing history).  It is trained by mean squared error against impulses the solver
produced, with Adam (Kingma & Ba, Algorithm 1: bias-corrected first and
second moments).  None of this is in the paper: it is the learned part added
on top of the method's warm start.

Parameter vector layout (shared with the C ABI): W1 [12][64] (input-major),
b1 [64], W2 [64][64], b2 [64], W3 [64][3], b3 [3]; 5187 values.

Plain numpy in float64: matrix products as library primitives, the backward
pass written out layer by layer.  Imported only by tests and the benchmark's
CPU-baseline leg.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 12, 64, 3
SHAPES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def relu(z):
    return np.maximum(z, 0.0)


def forward(theta, X):
    """Outputs [B][3] and the intermediate values the backward pass needs."""
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = relu(z1)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = relu(z2)
    y = X[:, 4:7] + h2 @ p["W3"] + p["b3"]
    return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2)


def loss(theta, X, T) -> float:
    """Mean over samples and outputs of the squared error."""
    y, _ = forward(theta, X)
    d = y - np.asarray(T, dtype=np.float64)
    return float(np.mean(d * d))


def grad(theta, X, T):
    """(loss, dloss/dtheta) by reverse-mode differentiation of ``loss``."""
    p = unpack(theta)
    y, c = forward(theta, X)
    T = np.asarray(T, dtype=np.float64)
    B = y.shape[0]
    d = y - T
    L = float(np.mean(d * d))
    dy = 2.0 * d / (B * N_OUT)                 # dL/dy
    g = {}
    g["W3"] = c["h2"].T @ dy
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"].T
    dz2 = dh2 * (c["z2"] > 0)
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (c["z1"] > 0)
    g["W1"] = c["X"].T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return L, pack(g)


def adam(theta, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1): returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def warm_start(theta, feat, scale, mu):
    """Impulses a trained network proposes for contacts: s*y, the normal one
    made non-negative and each friction one clamped to +-mu times it."""
    y, _ = forward(theta, feat)
    lam = y * np.asarray(scale, dtype=np.float64)[:, None]
    ln = np.maximum(lam[:, 0], 0.0)
    lim = np.asarray(mu, dtype=np.float64) * ln
    return np.stack([ln, np.clip(lam[:, 1], -lim, lim), np.clip(lam[:, 2], -lim, lim)], axis=1)
