"""Pins for the float64 MLP oracle: central finite differences, closed forms
for special weights, and the first Adam step."""
import numpy as np

from oracle import mlp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.he_init(rng) + rng.normal(0, 0.05, mlp.NPARAMS)   # nonzero biases too
    X = rng.normal(0, 1, (7, 4))
    t = rng.normal(0, 1, 7)
    g, _ = mlp.gradient(theta, X, t)
    h = 1e-6
    num = np.zeros_like(theta)
    for i in range(mlp.NPARAMS):
        e = np.zeros_like(theta)
        e[i] = h
        num[i] = (mlp.loss(theta + e, X, t) - mlp.loss(theta - e, X, t)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_zero_weights_closed_form():
    """All weights zero: the output is b3 everywhere, dL/db3 = 2*mean(b3 - t)
    and every other gradient vanishes (ReLU(0) = 0 and its slope at 0 is 0)."""
    theta = np.zeros(mlp.NPARAMS)
    theta[-1] = 0.7
    X = np.arange(12, dtype=float).reshape(3, 4)
    t = np.array([1.0, 2.0, -1.0])
    y, _ = mlp.forward(theta, X)
    assert np.all(y == 0.7)
    g, L = mlp.gradient(theta, X, t)
    assert np.isclose(g[-1], 2 * np.mean(0.7 - t))
    assert np.all(g[:-1] == 0)
    assert np.isclose(L, np.mean((0.7 - t) ** 2))


def test_linear_region_matches_matrix_product():
    """With positive inputs, weights and biases every ReLU is active, so the
    network is the plain product w3^T (W2 (W1 x + b1) + b2) + b3."""
    rng = np.random.default_rng(1)
    d = {"W1": rng.uniform(0.1, 1, (32, 4)), "b1": rng.uniform(0.1, 1, 32), "W2": rng.uniform(0.1, 1, (32, 32)),
         "b2": rng.uniform(0.1, 1, 32), "w3": rng.uniform(-1, 1, 32), "b3": np.array([0.3])}
    theta = mlp.pack(d)
    X = rng.uniform(0, 1, (5, 4))
    want = (d["W2"] @ (d["W1"] @ X.T + d["b1"][:, None]) + d["b2"][:, None]).T @ d["w3"] + 0.3
    y, _ = mlp.forward(theta, X)
    assert np.allclose(y, want, rtol=1e-13)


def test_first_adam_step_is_signed_lr():
    """After one Adam step from m = v = 0 the bias-corrected moments are g and
    g^2, so every parameter moves by -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 1, mlp.NPARAMS)
    g = rng.normal(0, 1, mlp.NPARAMS)
    new, m, v = mlp.adam_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    assert np.allclose(new - theta, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def test_features_formula():
    X = mlp.features([0, 10, 7], [0, 2, 7], [0, 6, 1])
    assert np.allclose(X[0], 0)
    assert np.allclose(X[1], np.log1p([10, 2, 6, 5]))
    assert np.allclose(X[2], np.log1p([7, 7, 1, 1]))
