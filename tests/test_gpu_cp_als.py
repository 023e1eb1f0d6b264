"""Eigenvalue-weighted CP-ALS of the projectors (Eqs. 15-16, App. I) on the GPU
against the float64 oracle (oracle/cp_als.py), from the same start point."""
import numpy as np
import pytest

from oracle import cp_als

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _case(o, v, N, W, seed, noise):
    rng = np.random.default_rng(seed)
    yo, yv, tau = (rng.standard_normal((n, W)) for n in (o, v, N))
    U = (yo[:, None, :] * yv[None, :, :]).reshape(o * v, W) @ tau.T
    U += noise * rng.standard_normal(U.shape)
    eps = rng.uniform(0.1, 3.0, N) * rng.choice([-1.0, 1.0], N)
    start = [a + 0.3 * rng.standard_normal(a.shape) for a in (yo, yv, tau)]
    return U, eps, start


@pytest.mark.parametrize("shape", [(4, 9, 7, 3, 1), (12, 40, 50, 24, 2), (7, 33, 65, 40, 3)],
                         ids=lambda s: "x".join(map(str, s)))
def test_cp_als_matches_oracle(shape):
    from paper_2111_11473_gb300 import binding
    o, v, N, W, seed = shape
    U, eps, start = _case(o, v, N, W, seed, noise=0.05)
    yo, yv, tau, hist = binding.cp_als(U, eps, *start, iters=6)
    ryo, ryv, rtau, rhist = cp_als.als(U, eps, *start, 6)
    assert np.allclose(hist, rhist, rtol=1e-9, atol=1e-12)
    rec = (yo[:, None, :] * yv[None, :, :]).reshape(o * v, W) @ tau.T
    rrec = (ryo[:, None, :] * ryv[None, :, :]).reshape(o * v, W) @ rtau.T
    assert np.abs(rec - rrec).max() < 1e-9 * max(1.0, np.abs(rrec).max())
    assert all(b <= a * (1 + 1e-10) for a, b in zip(hist, hist[1:]))


def test_cp_als_recovers_planted_projectors():
    from paper_2111_11473_gb300 import binding
    U, eps, start = _case(6, 30, 20, 10, 5, noise=0.0)
    _, _, _, hist = binding.cp_als(U, eps, *start, iters=80)
    assert hist[-1] < 1e-14 * float(np.sum((eps[None, :] * U) ** 2))
