"""Spin-orbital CCSD residual (Stanton-Gauss intermediates).

Test infrastructure only (see the package docstring).

An independent formulation of CCSD that shares nothing with the closed-shell
T1-dressed residual of ``closed_shell``: antisymmetrised spin-orbital
integrals, no T1 dressing, explicit singles terms (J. F. Stanton, J. Gauss,
J. D. Watts, R. J. Bartlett, J. Chem. Phys. 94, 4334 (1991)).  For a
closed-shell reference the alpha-beta block of its doubles residual and the
alpha block of its singles residual equal the closed-shell residual that the
paper builds on (its ref. 107), so it pins that algebra.

Spin-orbital index P = 2 p + s (s = 0 alpha, 1 beta); occupied spin
orbitals 0..2o-1 come first.
"""
from __future__ import annotations

import numpy as np


def _es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


def spin_blocks(h, g, o):
    """Fock matrix and antisymmetrised <pq||rs> in the spin-orbital basis.

    h: (n, n) core Hamiltonian, g: (n, n, n, n) Mulliken (pq|rs).
    Returns f (2n, 2n) and the <pq||rs> tensor (2n)^4, physicists' order.
    """
    n = h.shape[0]
    spin = np.arange(2 * n) % 2
    spat = np.arange(2 * n) // 2
    same = (spin[:, None] == spin[None, :]).astype(float)
    hso = h[np.ix_(spat, spat)] * same
    # Mulliken (PQ|RS) = (pq|rs) d(sP,sQ) d(sR,sS)
    gso = g[np.ix_(spat, spat, spat, spat)] * same[:, :, None, None] * same[None, None, :, :]
    phys = gso.transpose(0, 2, 1, 3)          # <PR|QS> -> <pq|rs> = (pr|qs)
    anti = phys - phys.transpose(0, 1, 3, 2)
    nocc = 2 * o
    f = hso + _es('pkqk->pq', anti[:, :nocc, :, :nocc])
    return f, anti


def to_spin_amplitudes(t1, t2):
    """Closed-shell t1[i,a], t2[i,j,a,b] -> spin-orbital amplitudes.

    t(I s, A s') = d(s,s') t_i^a;
    t(I s, J t, A s', B t') = d(s,s')d(t,t') t_ij^ab - d(s,t')d(t,s') t_ij^ba.
    """
    o, v = t1.shape
    so = np.arange(2 * o)
    sv = np.arange(2 * v)
    si, pi = so % 2, so // 2
    sa, pa = sv % 2, sv // 2
    T1 = t1[np.ix_(pi, pa)] * (si[:, None] == sa[None, :])
    d = lambda x, y: (x[:, None] == y[None, :]).astype(float)
    tab = t2[np.ix_(pi, pi, pa, pa)]
    tba = t2.transpose(0, 1, 3, 2)[np.ix_(pi, pi, pa, pa)]
    T2 = (tab * d(si, sa)[:, None, :, None] * d(si, sa)[None, :, None, :]
          - tba * d(si, sa)[:, None, None, :] * d(si, sa)[None, :, :, None])
    return T1, T2


def residual(f, w, T1, T2, nocc):
    """Spin-orbital CCSD residual (R1[I,A], R2[I,J,A,B]).

    The full Fock matrix (diagonal included) enters the F intermediates, so
    the returned arrays are <Phi_I^A|Hbar|0> and <Phi_IJ^AB|Hbar|0>.
    """
    o = slice(0, nocc)
    v = slice(nocc, f.shape[0])
    fov, foo, fvv = f[o, v], f[o, o], f[v, v]
    t1, t2 = T1, T2
    tau_t = t2 + 0.5 * (_es('ia,jb->ijab', t1, t1) - _es('ib,ja->ijab', t1, t1))
    tau = t2 + _es('ia,jb->ijab', t1, t1) - _es('ib,ja->ijab', t1, t1)

    Fae = (fvv - 0.5 * _es('me,ma->ae', fov, t1)
           + _es('mf,mafe->ae', t1, w[o, v, v, v])
           - 0.5 * _es('mnaf,mnef->ae', tau_t, w[o, o, v, v]))
    Fmi = (foo + 0.5 * _es('ie,me->mi', t1, fov)
           + _es('ne,mnie->mi', t1, w[o, o, o, v])
           + 0.5 * _es('inef,mnef->mi', tau_t, w[o, o, v, v]))
    Fme = fov + _es('nf,mnef->me', t1, w[o, o, v, v])

    Wmnij = (w[o, o, o, o]
             + _es('je,mnie->mnij', t1, w[o, o, o, v])
             - _es('ie,mnje->mnij', t1, w[o, o, o, v])
             + 0.25 * _es('ijef,mnef->mnij', tau, w[o, o, v, v]))
    Wabef = (w[v, v, v, v]
             - _es('mb,amef->abef', t1, w[v, o, v, v])
             + _es('ma,bmef->abef', t1, w[v, o, v, v])
             + 0.25 * _es('mnab,mnef->abef', tau, w[o, o, v, v]))
    Wmbej = (w[o, v, v, o]
             + _es('jf,mbef->mbej', t1, w[o, v, v, v])
             - _es('nb,mnej->mbej', t1, w[o, o, v, o])
             - _es('jnfb,mnef->mbej', 0.5 * t2 + _es('jf,nb->jnfb', t1, t1),
                   w[o, o, v, v]))

    r1 = (fov.copy()
          + _es('ie,ae->ia', t1, Fae)
          - _es('ma,mi->ia', t1, Fmi)
          + _es('imae,me->ia', t2, Fme)
          - _es('nf,naif->ia', t1, w[o, v, o, v])
          - 0.5 * _es('imef,maef->ia', t2, w[o, v, v, v])
          - 0.5 * _es('mnae,nmei->ia', t2, w[o, o, v, o]))

    r2 = w[o, o, v, v].copy()
    tmp = _es('ijae,be->ijab', t2, Fae - 0.5 * _es('mb,me->be', t1, Fme))
    r2 += tmp - tmp.transpose(0, 1, 3, 2)
    tmp = _es('imab,mj->ijab', t2, Fmi + 0.5 * _es('je,me->mj', t1, Fme))
    r2 -= tmp - tmp.transpose(1, 0, 2, 3)
    r2 += 0.5 * _es('mnab,mnij->ijab', tau, Wmnij)
    r2 += 0.5 * _es('ijef,abef->ijab', tau, Wabef)
    tmp = (_es('imae,mbej->ijab', t2, Wmbej)
           - _es('ie,ma,mbej->ijab', t1, t1, w[o, v, v, o]))
    r2 += (tmp - tmp.transpose(1, 0, 2, 3) - tmp.transpose(0, 1, 3, 2)
           + tmp.transpose(1, 0, 3, 2))
    tmp = _es('ie,abej->ijab', t1, w[v, v, v, o])
    r2 += tmp - tmp.transpose(1, 0, 2, 3)
    tmp = _es('ma,mbij->ijab', t1, w[o, v, o, o])
    r2 -= tmp - tmp.transpose(0, 1, 3, 2)
    return r1, r2


def energy(f, w, T1, T2, nocc):
    """E = sum f_ia t_i^a + 1/4 <ij||ab> t_ij^ab + 1/2 <ij||ab> t_i^a t_j^b."""
    o = slice(0, nocc)
    v = slice(nocc, f.shape[0])
    return float(_es('ia,ia->', f[o, v], T1)
                 + 0.25 * _es('ijab,ijab->', w[o, o, v, v], T2)
                 + 0.5 * _es('ijab,ia,jb->', w[o, o, v, v], T1, T1))


def closed_shell_view(R1, R2):
    """alpha singles block [i, a] and alpha-beta doubles block [i, j, a, b]."""
    return R1[0::2, 0::2], R2[0::2, 1::2, 0::2, 1::2]
