"""FP64 reference of the ordering MLP (TEST INFRASTRUCTURE ONLY).

Network: y = w2 . relu(W1 x + b1) + b2 with x in R^256, W1 in R^{256x256},
b1, w2 in R^256, b2 in R; loss = mean_r (y_r - target_r)^2.

The GPU forward multiplies bfloat16 copies of x and W1 (fp32 accumulate);
these functions take whatever (already rounded) values they are given and
compute in float64, so comparing the GPU against forward/backward on the same
rounded inputs isolates the accumulation error.  backward() is the
hand-derived chain rule; tests pin it with central finite differences of
loss().
"""

from __future__ import annotations

import numpy as np


def forward(W1, b1, w2, b2, X):
    W1 = np.asarray(W1, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    Z = X @ W1.T + np.asarray(b1, dtype=np.float64)
    H = np.maximum(Z, 0.0)
    y = H @ np.asarray(w2, dtype=np.float64) + float(b2)
    return Z, H, y


def loss(W1, b1, w2, b2, X, target):
    _, _, y = forward(W1, b1, w2, b2, X)
    d = y - np.asarray(target, dtype=np.float64)
    return float(np.mean(d * d))


def backward(W1, b1, w2, b2, X, target):
    """Gradients of loss() w.r.t. (W1, b1, w2, b2)."""
    X = np.asarray(X, dtype=np.float64)
    Z, H, y = forward(W1, b1, w2, b2, X)
    B = X.shape[0]
    dy = 2.0 * (y - np.asarray(target, dtype=np.float64)) / B
    dw2 = H.T @ dy
    db2 = float(dy.sum())
    dH = np.outer(dy, np.asarray(w2, dtype=np.float64))
    dZ = dH * (Z > 0)
    db1 = dZ.sum(axis=0)
    dW1 = dZ.T @ X
    return dW1, db1, dw2, db2
