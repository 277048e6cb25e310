"""FP64 reference of the schedule MLP (6 -> 32 -> 32 -> 1, ReLU): forward
pass, mean-squared loss and its gradient, written from the definitions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Parameter layout, flat:
W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3.
"""
from __future__ import annotations

import numpy as np

H, NIN = 32, 6
NPARAM = H * NIN + H + H * H + H + H + 1


def unpack(w: np.ndarray):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + H * NIN].reshape(H, NIN); o += H * NIN
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o]
    return W1, b1, W2, b2, W3, b3


def forward(w, X):
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    return h2 @ W3 + b3


def loss(w, X, Y):
    e = forward(w, X) - np.asarray(Y, dtype=np.float64)
    return float(np.mean(e * e))


def grad(w, X, Y):
    """Gradient of loss() by the chain rule (backpropagation)."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    gy = 2.0 * (y - np.asarray(Y, dtype=np.float64)) / N
    gW3 = h2.T @ gy
    gb3 = gy.sum()
    dz2 = np.outer(gy, W3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
