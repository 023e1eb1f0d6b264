"""Pins of the FP64 reference network of the learned preconditioner.

Its hand-written backward pass is checked against central finite differences
of its loss (an independent route to the gradient), and one Adam step
against the update rule written out.
"""
import numpy as np

from oracle import mlp


def _data(n, F, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, F))
    j = rng.standard_normal(n)
    t = j * (1 + 0.3 * np.tanh(X[:, 0])) + 0.05 * rng.standard_normal(n)
    return X, j, t


def test_backward_matches_finite_differences():
    F, H = 8, 12
    th = mlp.init(F, H, 3)
    rng = np.random.default_rng(4)
    th += 0.1 * rng.standard_normal(th.shape)       # non-zero output layer too
    X, j, t = _data(40, F, 5)
    L, g = mlp.grad(th, X, j, t, F, H)
    assert abs(L - mlp.loss(th, X, j, t, F, H)) < 1e-15
    h = 1e-6
    idx = rng.choice(th.size, 60, replace=False)
    for k in idx:
        e = np.zeros_like(th)
        e[k] = h
        fd = (mlp.loss(th + e, X, j, t, F, H) - mlp.loss(th - e, X, j, t, F, H)) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(g[k]))


def test_untrained_network_is_plain_jacobi():
    F, H = 8, 16
    th = mlp.init(F, H, 0)
    X, j, t = _data(10, F, 1)
    y, _ = mlp.forward(th, X, F, H)
    assert np.all(y == 0.0)                     # zero output layer: factor 1


def test_adam_step_closed_form():
    th = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    th1, m1, v1 = mlp.adam_step(th, g, m, v, 1, 0.1)
    # first step with bias correction moves every coordinate by lr * sign(g)
    assert np.allclose(th1, th - 0.1 * np.sign(g), atol=1e-7)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
