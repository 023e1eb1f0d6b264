"""Jacobi + DIIS drivers for canonical and THC-projected CCSD.

Test infrastructure only (see the package docstring).

The paper states only that the residual is converged to 1e-8 (Fig. 3
caption); the update used here is the orbital-energy Jacobi step with Pulay
DIIS:
  canonical:  t1 -= Omega1 / (eps_a - eps_i),  t2 -= Omega2 / D_ij^ab;
  projected:  T  -= sigma_q / (e_P + e_Q),     t1 as above,
where sigma_q = C^T sigma C in the orthonormal basis of Eq. 22 (T^PQ, the
working variable the paper recommends) and e are the generalised eigenvalues
of (F_eps, S), so e_P + e_Q is exactly the Fock part of the projected
Jacobian.  Convergence: sqrt(|Omega1|^2 + |residual of the doubles|^2) < tol.
"""
from __future__ import annotations

import numpy as np

from . import closed_shell as cs
from . import thc


class DIIS:
    """Pulay DIIS on (vector, error) pairs; keeps the last ``size`` pairs."""

    def __init__(self, size=8):
        self.size = size
        self.x = []
        self.e = []

    def push(self, x, e):
        self.x.append(x.copy())
        self.e.append(e.copy())
        if len(self.x) > self.size:
            self.x.pop(0)
            self.e.pop(0)

    def extrapolate(self):
        m = len(self.x)
        if m < 2:
            return self.x[-1]
        B = np.zeros((m + 1, m + 1))
        E = np.array(self.e)
        B[:m, :m] = E @ E.T
        B[:m, m] = B[m, :m] = -1.0
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
        return np.tensordot(c, np.array(self.x), axes=1)


def solve_canonical(H: cs.Hamiltonian, eps_o, eps_v, tol=1e-8, max_iter=200,
                    diis_size=8):
    """Canonical closed-shell CCSD.  Returns (E, t1, t2, iters)."""
    o, v = H.o, H.v
    d1 = eps_v[None, :] - eps_o[:, None]
    d2 = d1[:, None, :, None] + d1[None, :, None, :]
    t1 = np.zeros((o, v))
    t2 = np.zeros((o, o, v, v))
    diis = DIIS(diis_size)
    for it in range(1, max_iter + 1):
        r1, r2 = cs.residual(H, t1, t2)
        norm = np.sqrt(np.sum(r1 ** 2) + np.sum(r2 ** 2))
        if norm < tol:
            return cs.energy(H, t1, t2), t1, t2, it
        step = np.concatenate([(-r1 / d1).ravel(), (-r2 / d2).ravel()])
        x = np.concatenate([t1.ravel(), t2.ravel()]) + step
        diis.push(x, step)
        x = diis.extrapolate()
        t1 = x[:o * v].reshape(o, v)
        t2 = x[o * v:].reshape(o, o, v, v)
        t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    raise RuntimeError(f"canonical CCSD not converged, |r| = {norm:.3e}")


def projected_residual(H: cs.Hamiltonian, Y, Zc, t1):
    """(sigma1[i,a], sigma[W,X]) of THC-RR-CCSD at (Zc, t1)."""
    t2 = thc.amplitudes(Y, Zc, H.o)
    r1, r2 = cs.residual(H, t1, t2)
    return r1, thc.project(Y, r2, H.o)


def solve_thc(H: cs.Hamiltonian, Y, eps_o, eps_v, tol=1e-8, max_iter=200,
              diis_size=8, rel_cut=1e-10, history=None):
    """THC-RR-CCSD.  Returns (E, Zc, t1, iters)."""
    o, v = H.o, H.v
    C, e = thc.metric_basis(Y, eps_o, eps_v, rel_cut)
    r = e.shape[0]
    dq = e[:, None] + e[None, :]
    d1 = eps_v[None, :] - eps_o[:, None]
    T = np.zeros((r, r))
    t1 = np.zeros((o, v))
    diis = DIIS(diis_size)
    for it in range(1, max_iter + 1):
        Zc = C @ T @ C.T
        r1, sig = projected_residual(H, Y, Zc, t1)
        sq = C.T @ sig @ C
        norm = np.sqrt(np.sum(r1 ** 2) + np.sum(sq ** 2))
        if history is not None:
            t2 = thc.amplitudes(Y, Zc, o)
            history.append((cs.energy(H, t1, t2), norm))
        if norm < tol:
            t2 = thc.amplitudes(Y, Zc, o)
            return cs.energy(H, t1, t2), Zc, t1, it
        step = np.concatenate([(-r1 / d1).ravel(), (-sq / dq).ravel()])
        x = np.concatenate([t1.ravel(), T.ravel()]) + step
        diis.push(x, step)
        x = diis.extrapolate()
        t1 = x[:o * v].reshape(o, v)
        T = x[o * v:].reshape(r, r)
        T = 0.5 * (T + T.T)
    raise RuntimeError(f"THC-RR-CCSD not converged, |r| = {norm:.3e}")


def mp2_energy(H: cs.Hamiltonian, eps_o, eps_v):
    """Closed-shell MP2 energy with the Cholesky ovov integrals."""
    g = H.g_ovov_chol
    d = (eps_o[:, None, None, None] - eps_v[None, :, None, None]
         + eps_o[None, None, :, None] - eps_v[None, None, None, :])
    return float(np.sum(g * (2.0 * g - g.transpose(0, 3, 2, 1)) / d))
