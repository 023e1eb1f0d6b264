"""Integrals for the oracle: T1 dressing, ERI blocks, Fock matrices.

Test infrastructure only (see the package docstring).

Conventions: MO index p runs over occupied (0..o-1) then virtual (o..n-1);
Cholesky vectors L[K, p, q] with (pq|rs) = sum_K L[K,p,q] L[K,r,s]  (Eq. 24).
Singles t1[i, a] = t_i^a.  All arithmetic in float64.
"""
from __future__ import annotations

import numpy as np


def t1_matrix(t1: np.ndarray, n: int) -> np.ndarray:
    """n x n matrix whose only non-zero block is [a, i] = t_i^a."""
    o, v = t1.shape
    m = np.zeros((n, n))
    m[o:, :o] = t1.T
    return m


def dress_cholesky(L: np.ndarray, t1: np.ndarray) -> np.ndarray:
    """T1-transformed Cholesky vectors, Eqs. 25-27 in the MO basis (C = 1).

    Eq. 25 gives C^p = 1 - tau^T and Eq. 26 gives C^h = 1 + tau^T with
    tau[i, a] = t_i^a, so  L^_pq = sum_rs C^p_rp C^h_sq L_rs.
    """
    n = L.shape[1]
    tau_T = t1_matrix(t1, n)          # [a, i] = t_i^a, i.e. tau^T
    Cp = np.eye(n) - tau_T.T          # C^p_{r p}: column a gets -t_i^a at row i
    Ch = np.eye(n) + tau_T            # C^h_{s q}: column i gets +t_i^a at row a
    return np.einsum('rp,Krs,sq->Kpq', Cp, L, Ch, optimize=True)


def eri(La: np.ndarray, Lb: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum_K La[K,p,q] Lb[K,r,s]  (Eq. 24)."""
    return np.einsum('Kpq,Krs->pqrs', La, Lb, optimize=True)


def thc_ovov(x: np.ndarray, z: np.ndarray, o: int) -> np.ndarray:
    """(ia|jb) = sum_IJ x_i^I x_a^I z^IJ x_j^J x_b^J  (Eq. 17)."""
    xo, xv = x[:o], x[o:]
    return np.einsum('iI,aI,IJ,jJ,bJ->iajb', xo, xv, z, xo, xv, optimize=True)


def core_hamiltonian(L: np.ndarray, eps_o: np.ndarray, eps_v: np.ndarray) -> np.ndarray:
    """One-electron h such that the Fock matrix is diag(eps).

    The paper gives no core Hamiltonian; canonical Hartree-Fock orbitals are
    assumed, f = diag(eps_o, eps_v), and h is recovered from
    f_pq = h_pq + sum_k [2 (pq|kk) - (pk|kq)].
    """
    o = eps_o.shape[0]
    f = np.diag(np.concatenate([eps_o, eps_v]))
    g_pqkk = np.einsum('Kpq,Kkk->pq', L, L[:, :o, :o])
    g_pkkq = np.einsum('Kpk,Kkq->pq', L[:, :, :o], L[:, :o, :])
    return f - (2.0 * g_pqkk - g_pkkq)


def dressed_fock(h: np.ndarray, L: np.ndarray, t1: np.ndarray, o: int) -> np.ndarray:
    """F^_pq = h^_pq + sum_k [2 (pq^|kk) - (pk^|kq)]  with h^ and L^ T1-dressed."""
    n = h.shape[0]
    tau_T = t1_matrix(t1, n)
    Cp = np.eye(n) - tau_T.T
    Ch = np.eye(n) + tau_T
    hh = Cp.T @ h @ Ch
    Lh = dress_cholesky(L, t1)
    J = np.einsum('Kpq,Kkk->pq', Lh, Lh[:, :o, :o])
    Kx = np.einsum('Kpk,Kkq->pq', Lh[:, :, :o], Lh[:, :o, :])
    return hh + 2.0 * J - Kx
