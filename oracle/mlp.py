"""FP64 reference of the planner's cost-model MLP.

TEST INFRASTRUCTURE ONLY (imported by tests; the engine never imports it).

Network: y = w3 . ReLU(W2^T ReLU(W1^T xn + b1) + b2) + b3 with xn = (x - mean)
/ std, parameters flattened as W1[in][h] b1[h] W2[h][h] b2[h] w3[h] b3.  Loss:
mean over the batch of (y - t)^2.  The gradient is the textbook chain rule,
written out layer by layer; the tests pin it to central finite differences.
"""
from __future__ import annotations

import numpy as np


def unpack(p: np.ndarray, n_in: int, h: int):
    p = np.asarray(p, np.float64)
    o = 0
    W1 = p[o:o + n_in * h].reshape(n_in, h); o += n_in * h
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    w3 = p[o:o + h]; o += h
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, x, mean, std, n_in, h):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, h)
    xn = (np.asarray(x, np.float64) - mean) / std
    a1 = xn @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    return y, (xn, a1, h1, a2, h2)


def loss_and_grad(p, x, t, mean, std, n_in, h):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, h)
    y, (xn, a1, h1, a2, h2) = forward(p, x, mean, std, n_in, h)
    B = len(y)
    e = y - np.asarray(t, np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B                      # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = np.sum(dy)
    dh2 = np.outer(dy, w3) * (a2 > 0)     # through ReLU
    g_W2 = h1.T @ dh2
    g_b2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2.T) * (a1 > 0)
    g_W1 = xn.T @ dh1
    g_b1 = dh1.sum(axis=0)
    grad = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, grad


def n_params(n_in: int, h: int) -> int:
    return n_in * h + h + h * h + h + h + 1
