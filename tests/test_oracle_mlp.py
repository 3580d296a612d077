"""Pins of the oracle's warm-start network: its backward pass against central finite
differences (FP64), and Adam against its closed form on a quadratic."""
import numpy as np

from oracle import taps_oracle as O


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    dims = [5, 7, 6, 3]
    n = sum(i * o + o for i, o in zip(dims[:-1], dims[1:]))
    p = rng.normal(0, 0.5, n)
    X = rng.normal(0, 1, (4, 5))
    T = rng.normal(0, 1, (4, 3))
    loss, g = O.mlp_loss_grad(p, dims, X, T)
    h = 1e-6
    fd = np.zeros(n)
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        fd[k] = (O.mlp_loss_grad(p + e, dims, X, T)[0] - O.mlp_loss_grad(p - e, dims, X, T)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) < 1e-6 * max(1.0, np.max(np.abs(g)))


def test_linear_network_gradient_closed_form():
    """No hidden layer: loss = mean((X W^T + b - T)^2), dW = 2/n (Y-T)^T X."""
    rng = np.random.default_rng(1)
    dims = [3, 2]
    p = rng.normal(size=3 * 2 + 2)
    X, T = rng.normal(size=(5, 3)), rng.normal(size=(5, 2))
    W, b = p[:6].reshape(2, 3), p[6:]
    Y = X @ W.T + b
    _, g = O.mlp_loss_grad(p, dims, X, T)
    assert np.allclose(g[:6].reshape(2, 3), 2.0 / Y.size * (Y - T).T @ X)
    assert np.allclose(g[6:], 2.0 / Y.size * (Y - T).sum(axis=0))


def test_adam_first_step_moves_by_lr():
    """At t = 1 the bias-corrected step is lr * g / (|g| + eps) = lr * sign(g)."""
    g = np.array([3.0, -0.5, 1e-3])
    p1, m, v = O.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(p1, -0.01 * np.sign(g))
