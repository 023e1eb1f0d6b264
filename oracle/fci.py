"""Two-electron full configuration interaction (singlet).

Test infrastructure only (see the package docstring).

For two electrons CCSD is exact, so with one doubly occupied orbital the
converged CCSD energy must equal the lowest singlet FCI energy.  The singlet
spatial wavefunction is Psi(1,2) = sum_pq c_pq phi_p(1) phi_q(2) with c
symmetric; H = h(1) + h(2) + 1/r12 acts as
  <pq|H|rs> = h_pr d_qs + d_pr h_qs + (pr|qs).
"""
from __future__ import annotations

import numpy as np


def singlet_ground_energy(h: np.ndarray, g: np.ndarray) -> float:
    """Lowest singlet eigenvalue; h (n,n), g (n,n,n,n) Mulliken."""
    n = h.shape[0]
    eye = np.eye(n)
    H = (np.einsum('pr,qs->pqrs', h, eye) + np.einsum('pr,qs->pqrs', eye, h)
         + g.transpose(0, 2, 1, 3)).reshape(n * n, n * n)
    cols = []
    for p in range(n):
        for q in range(p, n):
            c = np.zeros((n, n))
            c[p, q] += 1.0
            c[q, p] += 1.0
            cols.append(c.ravel() / np.linalg.norm(c))
    B = np.array(cols).T
    Hs = B.T @ H @ B
    return float(np.linalg.eigvalsh(0.5 * (Hs + Hs.T))[0])
