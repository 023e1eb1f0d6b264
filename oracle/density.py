"""MP2-like one-particle density matrices from doubles amplitudes.

Test infrastructure only (see the package docstring).

App. II, Eqs. 47-48 (closed shell, both spins summed):
    D_ij = -2 sum_kab t_ik^ab [2 t_jk^ab - t_jk^ba]
    D_ab =  2 sum_ijc t_ij^ac [2 t_ij^bc - t_ji^bc]
evaluated on the full 4-index amplitudes (the definitions written out; the
paper's O(N^4) THC factorisation, Eqs. 49-56, is what the GPU library
implements).  ``spin_orbital_density`` is the textbook spin-orbital form
D_IJ = -1/2 sum_KAB t_IK^AB t_JK^AB, D_AB = 1/2 sum_IJC t_IJ^AC t_IJ^BC, used
to pin the closed-shell expressions.
"""
from __future__ import annotations

import numpy as np


def _es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


def mp2_density(t2):
    """(D_oo, D_vv) of Eqs. 47-48 from t2[i, j, a, b]."""
    u = 2.0 * t2 - t2.transpose(0, 1, 3, 2)            # 2 t_jk^ab - t_jk^ba
    Doo = -2.0 * _es('ikab,jkab->ij', t2, u)
    w = 2.0 * t2 - t2.transpose(1, 0, 2, 3)            # 2 t_ij^bc - t_ji^bc
    Dvv = 2.0 * _es('ijac,ijbc->ab', t2, w)
    return Doo, Dvv


def spin_orbital_density(T2, nocc):
    """Spin-orbital (D_IJ, D_AB) from antisymmetric amplitudes T2[I, J, A, B]."""
    Doo = -0.5 * _es('ikab,jkab->ij', T2, T2)
    Dvv = 0.5 * _es('ijac,ijbc->ab', T2, T2)
    return Doo, Dvv
