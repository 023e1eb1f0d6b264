"""The learned preconditioner's GPU kernels against the FP64 reference network."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

F = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, F)).astype(np.float32)
    j = rng.standard_normal(n).astype(np.float32)
    t = (j * (1 + 0.3 * np.tanh(X[:, 0])) + 0.05 * rng.standard_normal(n)).astype(np.float32)
    return X, j, t


def _params(H, seed):
    th = omlp.init(F, H, seed)
    th += 0.05 * np.random.default_rng(seed + 1).standard_normal(th.shape)
    return th


@pytest.mark.parametrize("H", [32, 256])
def test_float32_gradient_matches_reference(H):
    import paper_2111_11473_gb300 as pkg
    th = _params(H, 7)
    X, j, t = _data(700, 8)
    net = pkg.Mlp(hidden=H, bf16=False)
    net.set_params(th.astype(np.float32))
    L, g = net.loss_grad(X, j, t)
    th32 = th.astype(np.float32).astype(np.float64)
    Lr, gr = omlp.grad(th32, X.astype(np.float64), j.astype(np.float64), t.astype(np.float64), F, H)
    assert abs(L - Lr) < 1e-5 * Lr
    # float32 accumulation over 700 samples: 1e-4 of the largest gradient entry
    assert np.abs(g - gr).max() < 1e-4 * np.abs(gr).max()
    y = net.predict(X)
    yr, _ = omlp.forward(th32, X.astype(np.float64), F, H)
    assert np.abs(y - yr).max() < 1e-5 * max(1.0, np.abs(yr).max())
    net.close()


def test_bf16_forward_within_bound():
    """bf16 weights/activations in the H x H layer: 2^-8 per factor, H = 256 terms."""
    import paper_2111_11473_gb300 as pkg
    H = 256
    th = _params(H, 9)
    X, j, t = _data(1000, 10)
    net = pkg.Mlp(hidden=H, bf16=True)
    net.set_params(th.astype(np.float32))
    y = net.predict(X)
    yr, _ = omlp.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float64), F, H)
    err = np.abs(y - yr).max() / max(1e-3, np.abs(yr).max())
    print(f"bf16 forward: max rel err {err:.2e}")
    assert err < 2e-2
    net.close()


def test_adam_training_step_and_convergence():
    import paper_2111_11473_gb300 as pkg
    H = 64
    th = _params(H, 11)
    X, j, t = _data(512, 12)
    net = pkg.Mlp(hidden=H, bf16=False)
    net.set_params(th.astype(np.float32))
    # one epoch with one minibatch holding every sample = one Adam step
    net.train(X, j, t, epochs=1, batch=512, lr=1e-2, seed=3)
    th32 = th.astype(np.float32).astype(np.float64)
    _, g = omlp.grad(th32, X.astype(np.float64), j.astype(np.float64), t.astype(np.float64), F, H)
    ref, _, _ = omlp.adam_step(th32, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-2)
    got = net.get_params().astype(np.float64)
    # the first Adam step moves each weight by lr * sign(g) (up to eps)
    moved = np.abs(ref - th32) > 5e-3
    assert np.abs(got - ref)[moved].max() < 1e-4
    L0 = omlp.loss(th32, X.astype(np.float64), j.astype(np.float64), t.astype(np.float64), F, H)
    L1 = net.train(X, j, t, epochs=200, batch=128, lr=3e-3, seed=4)
    print(f"training loss {L0:.4f} -> {L1:.4f}")
    assert L1 < 0.2 * L0
    net.close()
