"""Float64 reference of the learned preconditioner's network.

Test infrastructure only (see the package docstring).  The GPU library
trains and runs the same network with its own kernels; this module is what
its forward values, gradients and Adam steps are checked against.  Its own
backward pass is pinned by central finite differences in the tests.

Network (pointwise over the elements of the working basis):
    z1 = W1 x + b1,  a1 = tanh(z1)          W1: H x F
    z2 = W2 a1 + b2, a2 = tanh(z2)          W2: H x H
    y  = w3 . a2 + b3                       w3: H
Loss over a batch of N samples (scaled Jacobi step j, scaled target t):
    L = (1/N) sum_n (j_n (1 + y_n) - t_n)^2
Parameters live in one flat vector [W1 | b1 | W2 | b2 | w3 | b3] (row-major).
"""
from __future__ import annotations

import numpy as np


def sizes(F: int, H: int):
    return [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)),
            ("b3", (1,))]


def n_params(F: int, H: int) -> int:
    return sum(int(np.prod(s)) for _, s in sizes(F, H))


def unpack(theta: np.ndarray, F: int, H: int):
    out, o = {}, 0
    for name, shape in sizes(F, H):
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def init(F: int, H: int, seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases, zero output layer (network = 0)."""
    rng = np.random.default_rng(seed)
    th = np.zeros(n_params(F, H))
    p = unpack(th, F, H)
    p["W1"][:] = rng.uniform(-1, 1, (H, F)) * np.sqrt(6.0 / (F + H))
    p["W2"][:] = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / (2 * H))
    return th


def forward(theta, X, F, H):
    p = unpack(theta, F, H)
    z1 = X @ p["W1"].T + p["b1"]
    a1 = np.tanh(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = np.tanh(z2)
    y = a2 @ p["w3"] + p["b3"][0]
    return y, (X, a1, a2)


def loss(theta, X, j, t, F, H):
    y, _ = forward(theta, X, F, H)
    r = j * (1.0 + y) - t
    return float(np.mean(r * r))


def grad(theta, X, j, t, F, H):
    """Loss and its gradient by the chain rule (flat vector)."""
    p = unpack(theta, F, H)
    y, (X, a1, a2) = forward(theta, X, F, H)
    N = X.shape[0]
    r = j * (1.0 + y) - t
    L = float(np.mean(r * r))
    dy = (2.0 / N) * r * j
    g = np.zeros_like(theta)
    q = unpack(g, F, H)
    q["w3"][:] = a2.T @ dy
    q["b3"][0] = dy.sum()
    dz2 = np.outer(dy, p["w3"]) * (1.0 - a2 * a2)
    q["W2"][:] = dz2.T @ a1
    q["b2"][:] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - a1 * a1)
    q["W1"][:] = dz1.T @ X
    q["b1"][:] = dz1.sum(0)
    return L, g


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
