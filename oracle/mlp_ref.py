"""fp64 reference of the cost-model network (TEST INFRASTRUCTURE ONLY).

The cost model predicts a variant's log run time from plan features, column
statistics and variant features; it replaces the paper's per-workload
heuristic optimizer (Section 8.3) with a per-query choice, which the paper
names as future work (Section 9.4).  The network is a plain multilayer
perceptron:

    xh = (x - mu) / sigma                      standardised features, F wide
    h1 = relu(xh @ W1 + b1)                    H hidden units
    h2 = relu(h1 @ W2 + b2)                    H hidden units
    y  = h2 @ w3 + b3                          predicted log time
    L  = mean((y - t)^2)                       mean squared error

trained with Adam (Kingma and Ba, 2015, Algorithm 1):

    m <- b1 m + (1 - b1) g ;  v <- b2 v + (1 - b2) g^2
    p <- p - lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps)

Parameters are one flat vector in the order W1 (F x H, row-major), b1 (H),
W2 (H x H), b2 (H), w3 (H), b3 (1): the layout the CUDA kernels use.
Plain numpy, float64, no blocking or fusion.
"""
from __future__ import annotations

import numpy as np


def n_params(F: int, H: int) -> int:
    return F * H + H + H * H + H + H + 1


def unpack(p: np.ndarray, F: int, H: int):
    o = 0
    W1 = p[o:o + F * H].reshape(F, H); o += F * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o:o + 1]; o += 1
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, np.ravel(b3)]).astype(np.float64)


def init(F: int, H: int, seed: int = 0) -> np.ndarray:
    """He-uniform initial weights, zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (F, H)) * np.sqrt(6.0 / F)
    W2 = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    w3 = rng.uniform(-1, 1, H) * np.sqrt(6.0 / H)
    return pack(W1, np.zeros(H), W2, np.zeros(H), w3, np.zeros(1))


def forward(p, X, mu, sigma, H: int):
    X = np.asarray(X, np.float64)
    F = X.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(p, np.float64), F, H)
    xh = (X - mu) / sigma
    z1 = xh @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3[0]
    return y, (xh, z1, h1, z2, h2)


def loss(y, t) -> float:
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def backward(p, cache, y, t, H: int) -> np.ndarray:
    """Gradient of the mean squared error with respect to the flat parameters
    (chain rule through the layers above, relu' = 1 where z > 0)."""
    xh, z1, h1, z2, h2 = cache
    B, F = xh.shape
    W1, b1, W2, b2, w3, b3 = unpack(np.asarray(p, np.float64), F, H)
    dy = 2.0 * (np.asarray(y, np.float64) - np.asarray(t, np.float64)) / B
    dw3 = h2.T @ dy
    db3 = np.array([dy.sum()])
    dz2 = np.outer(dy, w3) * (z2 > 0)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    dW1 = xh.T @ dz1
    db1 = dz1.sum(axis=0)
    return pack(dW1, db1, dW2, db2, dw3, db3)


def adam_step(p, g, m, v, k: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step number k >= 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
