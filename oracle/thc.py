"""THC amplitudes, projection of the residual, and the projector metric.

Test infrastructure only (see the package docstring).

  t_ij^ab = sum_WX y_i^W y_a^W Zc^WX y_j^X y_b^X                 (Eq. 23)
  sigma^WX = sum_ijab y_i^W y_a^W y_j^X y_b^X Omega_ij^ab         (Eq. 6 with
             the CP-factorised projector of Eq. 14 written in the y basis)
  S^WX = sum_ia y_i^W y_a^W y_i^X y_a^X                          (Eq. 10, tau = 1)

The orthonormal working basis of Eq. 22 (the paper recommends T^PQ there):
C solves F_eps C = S C diag(e), C^T S C = 1, where
F_eps^WX = sum_ia y_i^W y_a^W (eps_a - eps_i) y_i^X y_a^X.  Then
U~ = (y o y) C is semi-unitary (Eq. 12), Zc = C T C^T, sigma_q = C^T sigma C.
Eigen-directions of S below ``rel_cut * max`` are dropped (metric
pseudo-inverse).
"""
from __future__ import annotations

import numpy as np


def kr(y_o: np.ndarray, y_v: np.ndarray) -> np.ndarray:
    """Khatri-Rao projector U[(i,a), W] = y_i^W y_a^W, shape (o*v, P)."""
    o, P = y_o.shape
    v = y_v.shape[0]
    return (y_o[:, None, :] * y_v[None, :, :]).reshape(o * v, P)


def amplitudes(Y: np.ndarray, Zc: np.ndarray, o: int) -> np.ndarray:
    """Eq. 23: t2[i,j,a,b] from the THC core Zc."""
    y_o, y_v = Y[:o], Y[o:]
    return np.einsum('iW,aW,WX,jX,bX->ijab', y_o, y_v, Zc, y_o, y_v,
                     optimize=True)


def project(Y: np.ndarray, omega2: np.ndarray, o: int) -> np.ndarray:
    """sigma^WX = sum_ijab y_i^W y_a^W y_j^X y_b^X Omega_ij^ab."""
    y_o, y_v = Y[:o], Y[o:]
    return np.einsum('iW,aW,ijab,jX,bX->WX', y_o, y_v, omega2, y_o, y_v,
                     optimize=True)


def metric_basis(Y, eps_o, eps_v, rel_cut=1e-10):
    """Generalised eigenbasis (C, e) of (F_eps, S) on the range of S."""
    o = eps_o.shape[0]
    U = kr(Y[:o], Y[o:])
    d = (eps_v[None, :] - eps_o[:, None]).ravel()
    S = U.T @ U
    Fe = U.T @ (d[:, None] * U)
    s, V = np.linalg.eigh(S)
    keep = s > rel_cut * s.max()
    Xh = V[:, keep] / np.sqrt(s[keep])        # S^{-1/2} on the range of S
    e, W = np.linalg.eigh(Xh.T @ Fe @ Xh)
    return Xh @ W, e
