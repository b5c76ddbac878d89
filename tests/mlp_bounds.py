"""Tolerances for the network's BF16-operand, FP32-accumulate kernels
against the FP64 reference (oracle/mlp.py).

Error model: rounding to BF16 (8 significant bits, round to nearest) gives a
relative error spread roughly uniformly over [-u, u] with u = 2^-8, standard
deviation u / sqrt(3).  A sum of K products of rounded operands then has an
error of standard deviation sqrt(2/3) u sqrt(sum (a_k b_k)^2) from this
layer's roundings, plus sqrt(sum b_k^2 s_k^2) for errors s_k already in the
operands.  These standard deviations are propagated layer by layer (FP32
accumulation adds ~2^-24 relative, negligible), a ReLU whose pre-activation
lies within 6 standard deviations of zero may switch (its full term is
added), and the tolerance is 6 standard deviations plus a small absolute
floor.  A dropped term, a wrong sign, a transposed operand or a missing
ReLU mask moves results by the size of the term itself, far beyond this.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp as M

U = 2.0 ** -8
S_ROUND = U / np.sqrt(3.0)          # one rounding
S_PROD = U * np.sqrt(2.0 / 3.0)     # a product of two rounded operands
K_SIGMA = 6.0


def _rss(a2, w2):
    return np.sqrt(a2 @ w2)


def _forward_sigmas(theta, X, sX=None):
    p = M.unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    W1s, W2s, W3s = p["W1"] ** 2, p["W2"] ** 2, p["W3"] ** 2
    y, c = M.forward(theta, X)
    sX = np.zeros_like(X) if sX is None else np.asarray(sX, dtype=np.float64)
    sz1 = np.sqrt(_rss(sX ** 2, W1s) ** 2 + (S_PROD ** 2) * ((X ** 2) @ W1s))
    sh1 = np.where(c["z1"] > 0, np.sqrt(sz1 ** 2 + (S_ROUND * c["h1"]) ** 2), 0.0)
    sh1 = np.where(np.abs(c["z1"]) <= K_SIGMA * sz1, np.maximum(sh1, np.abs(c["z1"]) + sz1), sh1)
    sz2 = np.sqrt((sh1 ** 2) @ W2s + (S_PROD ** 2) * ((c["h1"] ** 2) @ W2s))
    sh2 = np.where(c["z2"] > 0, np.sqrt(sz2 ** 2 + (S_ROUND * c["h2"]) ** 2), 0.0)
    sh2 = np.where(np.abs(c["z2"]) <= K_SIGMA * sz2, np.maximum(sh2, np.abs(c["z2"]) + sz2), sh2)
    # the skip connection adds input features 4-6 (in FP32) to the outputs
    sy = np.sqrt((sh2 ** 2) @ W3s + (S_PROD ** 2) * ((c["h2"] ** 2) @ W3s) + sX[:, 4:7] ** 2)
    return y, c, dict(sX=sX, sz1=sz1, sh1=sh1, sz2=sz2, sh2=sh2, sy=sy)


def forward_tolerance(theta, X, sX=None):
    """Tolerance [B][3] on |y_kernel - y_ref|; sX: standard deviations of
    errors already in the inputs."""
    _, _, s = _forward_sigmas(theta, X, sX)
    return K_SIGMA * s["sy"] + 1e-6


def grad_tolerance(theta, X, T):
    """Tolerance [N_PARAMS] on |grad_kernel - grad_ref|."""
    p = M.unpack(theta)
    y, c, s = _forward_sigmas(theta, X)
    W2, W3 = p["W2"], p["W3"]
    B = y.shape[0]
    k = 2.0 / (B * M.N_OUT)
    dy = k * (y - np.asarray(T, dtype=np.float64))
    sdy = np.sqrt((k * s["sy"]) ** 2 + (S_ROUND * dy) ** 2)
    m2, m1 = c["z2"] > 0, c["z1"] > 0
    t2 = dy @ W3.T
    sdz2 = np.sqrt((sdy ** 2) @ (W3.T ** 2) + (S_PROD ** 2) * ((dy ** 2) @ (W3.T ** 2)) + (S_ROUND * t2) ** 2)
    sdz2 = np.where(m2, sdz2, 0.0)
    flip2 = np.abs(c["z2"]) <= K_SIGMA * s["sz2"]
    sdz2 = np.where(flip2, np.abs(t2) + sdz2, sdz2)
    dz2 = m2 * t2
    t1 = dz2 @ W2.T
    sdz1 = np.sqrt((sdz2 ** 2) @ (W2.T ** 2) + (S_PROD ** 2) * ((dz2 ** 2) @ (W2.T ** 2)) + (S_ROUND * t1) ** 2)
    sdz1 = np.where(m1, sdz1, 0.0)
    flip1 = np.abs(c["z1"]) <= K_SIGMA * s["sz1"]
    sdz1 = np.where(flip1, np.abs(t1) + sdz1, sdz1)
    dz1 = m1 * t1

    def wgrad(a, sa, b, sb):
        # sum over samples of a_i b_j with errors sa, sb in the operands
        return np.sqrt((sa ** 2).T @ (b ** 2) + (a ** 2).T @ (sb ** 2))

    X = c["X"]
    sx = np.sqrt(s["sX"] ** 2 + (S_ROUND * X) ** 2)
    g = {}
    g["W3"] = wgrad(c["h2"], s["sh2"], dy, sdy)
    g["b3"] = np.sqrt((sdy ** 2).sum(axis=0))
    g["W2"] = wgrad(c["h1"], s["sh1"], dz2, sdz2)
    g["b2"] = np.sqrt((sdz2 ** 2).sum(axis=0))
    g["W1"] = wgrad(X, sx, dz1, sdz1)
    g["b1"] = np.sqrt((sdz1 ** 2).sum(axis=0))
    return K_SIGMA * M.pack(g) + 1e-9
