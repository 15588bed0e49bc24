"""Float64 oracle of the nnz-prediction MLP (test infrastructure only).

The network maps 4 features of an output column -- log1p of flops_j, of
nnz(B(:,j)), of the largest and of the mean nnz(A(:,k)) over the k of B(:,j)
-- through two hidden layers of 32 ReLU units to one output, the prediction
of log1p(nnz(C(:,j))).  Loss: mean squared error.  Optimiser: Adam.

Parameters are one flat vector (the layout the CUDA kernels use):
    W1 (32 x 4, row = hidden unit) | b1 (32) | W2 (32 x 32) | b2 (32) | w3 (32) | b3 (1)
Only numpy; this module never touches the CUDA path.
"""
from __future__ import annotations

import numpy as np

H, F = 32, 4
SIZES = [("W1", H * F), ("b1", H), ("W2", H * H), ("b2", H), ("w3", H), ("b3", 1)]
NPARAMS = sum(s for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, s in SIZES:
        out[name] = theta[o:o + s]
        o += s
    out["W1"] = out["W1"].reshape(H, F)
    out["W2"] = out["W2"].reshape(H, H)
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def features(flops, nnzb, maxa):
    """log1p of (flops, nnz(B(:,j)), max nnz(A(:,k)), mean nnz(A(:,k))), the mean
    being flops / nnz(B(:,j)) (0 for an empty column)."""
    flops = np.asarray(flops, dtype=np.float64)
    nnzb = np.asarray(nnzb, dtype=np.float64)
    mean = np.where(nnzb > 0, flops / np.maximum(nnzb, 1), 0.0)
    return np.log1p(np.stack([flops, nnzb, np.asarray(maxa, dtype=np.float64), mean], axis=1))


def forward(theta, X):
    p = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(theta, X, t):
    y, _ = forward(theta, X)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(theta, X, t):
    """Analytic gradient of the mean squared error (backpropagation)."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["w3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return pack(g), float(np.mean((y - t) ** 2))


def adam_step(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); step counts from 1.  Returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def he_init(rng):
    """He-normal weights, zero biases."""
    d = {"W1": rng.normal(0, np.sqrt(2.0 / F), (H, F)), "b1": np.zeros(H),
         "W2": rng.normal(0, np.sqrt(2.0 / H), (H, H)), "b2": np.zeros(H),
         "w3": rng.normal(0, np.sqrt(2.0 / H), H), "b3": np.zeros(1)}
    return pack(d)
