"""Closed-shell T1-dressed CCSD residual on full 4-index tensors.

Test infrastructure only (see the package docstring).

The residual is written as the paper's per-term equations, each evaluated
plainly from its 4-index definition:

  doubles  Omega_ij^ab = Eq.29 + Eq.28 + Eq.31 + Eq.32 + Eq.33 + Eq.35 + Eq.41
  singles  Omega_i^a   = Eq.38 + Eq.42
  energy   closed-shell CCSD energy (Sec. II.a: "as usual in CCSD")

Readings of the printed equations (the tests against the independent
spin-orbital CCSD fix each one):
  * Eq. 31 and Eq. 38: integrals carry T1 dressing (the algorithms use the
    dressed vectors).
  * Eq. 35: the right-hand amplitude factor is 2 t_jl^bd - t_jl^db, and the
    prefactor is 1/2 (the spin-orbital pin fixes it).
  * Eq. 41: the symmetrisation is the (ia)<->(jb) pair swap,
      sum_c t_ij^ac Fb_bc + sum_c t_ji^bc Fb_ac
      - sum_k t_ik^ab Fb_kj - sum_k t_jk^ba Fb_ki,  Fb = F^ + xi.
Integral assignment follows the paper: the T2^2 terms of Eqs. 32, 33 and 35
use the THC ovov integrals (Eq. 17); every other term, the xi intermediates
(Eqs. 39-40) and the energy use the Cholesky integrals.

Array conventions: t2[i, j, a, b] = t_ij^ab, t1[i, a] = t_i^a,
ERIs in Mulliken order g[p, q, r, s] = (pq|rs).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import integrals as ints

EQ35_PREFACTOR = 0.5


def _es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


@dataclass
class Hamiltonian:
    """Everything the closed-shell residual needs, built once per system."""
    o: int
    v: int
    L: np.ndarray        # (K, n, n) Cholesky vectors
    h: np.ndarray        # (n, n) core Hamiltonian (backed out)
    g_ovov_thc: np.ndarray   # (o, v, o, v) THC ovov (ia|jb)
    g_ovov_chol: np.ndarray  # (o, v, o, v) Cholesky ovov (ia|jb)

    @classmethod
    def from_inputs(cls, eps_o, eps_v, L, x, z):
        o = eps_o.shape[0]
        v = eps_v.shape[0]
        h = ints.core_hamiltonian(L, eps_o, eps_v)
        gT = ints.thc_ovov(x, z, o)
        Lov = L[:, :o, o:]
        gC = ints.eri(Lov, Lov)
        return cls(o, v, L, h, gT, gC)


def u_amp(t2):
    """u_ij^ab = 2 t_ij^ab - t_ij^ba."""
    return 2.0 * t2 - t2.transpose(0, 1, 3, 2)


class Dressed:
    """Dressed ERI blocks and dressed Fock matrix for one t1."""

    def __init__(self, H: Hamiltonian, t1):
        o = H.o
        self.o = o
        self.Lh = ints.dress_cholesky(H.L, t1)
        self.F = ints.dressed_fock(H.h, H.L, t1, o)

    def g(self, blocks: str):
        """Dressed (pq^|rs) for a block pattern such as 'vovo'."""
        o = self.o
        sl = {'o': slice(0, o), 'v': slice(o, None)}
        a = self.Lh[:, sl[blocks[0]], sl[blocks[1]]]
        b = self.Lh[:, sl[blocks[2]], sl[blocks[3]]]
        return ints.eri(a, b)

    def Foo(self):
        return self.F[:self.o, :self.o]

    def Fvv(self):
        return self.F[self.o:, self.o:]

    def Fov(self):
        return self.F[:self.o, self.o:]

    def Fvo(self):
        return self.F[self.o:, :self.o]


# ---------------------------------------------------------------- doubles

def eq29(D: Dressed, t2):
    """Eq. 29: bare dressed (ai^|bj) plus the linear ring terms."""
    u = u_amp(t2)
    g_vovo = D.g('vovo')
    g_voov = D.g('voov')
    r = _es('aibj->ijab', g_vovo)
    r += _es('ikac,bjkc->ijab', u, g_voov)
    r += _es('jkbc,aikc->ijab', u, g_voov)
    return r


def eq28(D: Dressed, t2):
    """Eq. 28: particle-particle, hole-hole and mixed particle-hole ladders."""
    r = _es('ijcd,acbd->ijab', t2, D.g('vvvv'))
    r += _es('klab,kilj->ijab', t2, D.g('oooo'))
    r -= _es('ilcb,aclj->ijab', t2, D.g('vvoo'))
    r -= _es('kjad,kibd->ijab', t2, D.g('oovv'))
    return r


def eq31(D: Dressed, t2):
    """Eq. 31: remaining linear Omega^C terms, dressed (kj^|bc), (ki^|ac)."""
    g_oovv = D.g('oovv')
    r = -_es('ikac,kjbc->ijab', t2, g_oovv)
    r -= _es('jkbc,kiac->ijab', t2, g_oovv)
    return r


def eq32(H: Hamiltonian, t2):
    """Eq. 32: sum_kcld t_ij^cd t_kl^ab (kc|ld), THC (kc|ld)."""
    X = _es('ijcd,kcld->ijkl', t2, H.g_ovov_thc)
    return _es('ijkl,klab->ijab', X, t2)


def eq33(H: Hamiltonian, t2):
    """Eq. 33: sum_kcld t_ik^cb t_lj^ad (lc|kd), THC (lc|kd)."""
    X = _es('ikcb,lckd->ibld', t2, H.g_ovov_thc)
    return _es('ibld,ljad->ijab', X, t2)


def eq35(H: Hamiltonian, t2):
    """Eq. 35: quadratic ring term and removal of the spurious term."""
    g = H.g_ovov_thc
    u = u_amp(t2)
    Lg = 2.0 * g - g.transpose(0, 3, 2, 1)        # 2(kc|ld) - (kd|lc)
    X = _es('ikac,kcld->iald', u, Lg)
    r = _es('iald,jlbd->ijab', X, u)
    Y = _es('ikca,kdlc->iald', t2, g)
    r += _es('iald,jldb->ijab', Y, t2)
    return EQ35_PREFACTOR * r


def xi_oo(H: Hamiltonian, t2):
    """Eq. 39: xi_kj = sum_dem t_jm^de [2(me|kd) - (md|ke)], Cholesky ERIs."""
    g = H.g_ovov_chol
    return (2.0 * _es('jmde,mekd->kj', t2, g) - _es('jmde,mdke->kj', t2, g))


def xi_vv(H: Hamiltonian, t2):
    """Eq. 40: xi_bc = -sum_lmd t_lm^db [2(ld|mc) - (lc|md)], Cholesky ERIs."""
    g = H.g_ovov_chol
    return -(2.0 * _es('lmdb,ldmc->bc', t2, g) - _es('lmdb,lcmd->bc', t2, g))


def eq41(H: Hamiltonian, D: Dressed, t2):
    """Eq. 41: Fock and xi terms, symmetrised over the (ia)<->(jb) swap."""
    Fv = D.Fvv() + xi_vv(H, t2)
    Fo = D.Foo() + xi_oo(H, t2)
    r = _es('ijac,bc->ijab', t2, Fv)
    r += _es('jibc,ac->ijab', t2, Fv)
    r -= _es('ikab,kj->ijab', t2, Fo)
    r -= _es('jkba,ki->ijab', t2, Fo)
    return r


# ---------------------------------------------------------------- singles

def eq38(D: Dressed, t2):
    """Eq. 38: singles terms Omega^G and Omega^H (dressed integrals)."""
    g_ovvv = D.g('ovvv')
    r = 2.0 * _es('ikcd,kdac->ia', t2, g_ovvv) - _es('ikcd,kcad->ia', t2, g_ovvv)
    g_ovoo = D.g('ovoo')
    g_ooov = D.g('ooov')
    r -= 2.0 * _es('klac,lcki->ia', t2, g_ovoo) - _es('klac,likc->ia', t2, g_ooov)
    return r


def eq42(D: Dressed, t2):
    """Eq. 42: F^_ai + sum_kc (2 t_ik^ac - t_ik^ca) F^_kc."""
    return D.Fvo().T + _es('ikac,kc->ia', u_amp(t2), D.Fov())


# ---------------------------------------------------------------- totals

DOUBLES_TERMS = ("eq28", "eq29", "eq31", "eq32", "eq33", "eq35", "eq41")
SINGLES_TERMS = ("eq38", "eq42")


def residual_terms(H: Hamiltonian, t1, t2):
    """Every per-equation piece, as full tensors: {name: array}."""
    D = Dressed(H, t1)
    return {
        "eq28": eq28(D, t2),
        "eq29": eq29(D, t2),
        "eq31": eq31(D, t2),
        "eq32": eq32(H, t2),
        "eq33": eq33(H, t2),
        "eq35": eq35(H, t2),
        "eq41": eq41(H, D, t2),
        "eq38": eq38(D, t2),
        "eq42": eq42(D, t2),
    }


def residual(H: Hamiltonian, t1, t2):
    """Full closed-shell residual: (Omega1[i,a], Omega2[i,j,a,b])."""
    terms = residual_terms(H, t1, t2)
    r2 = sum(terms[k] for k in DOUBLES_TERMS)
    r1 = sum(terms[k] for k in SINGLES_TERMS)
    return r1, r2


def energy(H: Hamiltonian, t1, t2):
    """E = sum_iajb [2(ia|jb) - (ib|ja)] (t_ij^ab + t_i^a t_j^b), Cholesky ERIs."""
    g = H.g_ovov_chol
    tau = t2 + _es('ia,jb->ijab', t1, t1)
    return float(2.0 * _es('iajb,ijab->', g, tau) - _es('ibja,ijab->', g, tau))


def reference_energy(H: Hamiltonian):
    """Closed-shell determinant energy  sum_i (h_ii + f_ii)."""
    o = H.o
    L = H.L
    J = np.einsum('Kii,Kjj->', L[:, :o, :o], L[:, :o, :o])
    Kx = np.einsum('Kij,Kji->', L[:, :o, :o], L[:, :o, :o])
    return float(2.0 * np.trace(H.h[:o, :o]) + 2.0 * J - Kx)
