"""Pins of the FP64 oracle against results fixed by theory, not by itself.

* closed-shell residual == alpha-beta block of an independent spin-orbital
  CCSD (Stanton-Gauss), at arbitrary t1, t2 (all terms, all T1 dressing);
* two-electron CCSD == two-electron full CI (CCSD is exact there);
* one Jacobi step from zero gives the closed-form MP2 energy;
* full THC rank (P = o v, generic Y) reproduces canonical CCSD;
* symmetry, polynomial degree and gauge invariance of the projected residual;
* planted mistakes in the oracle are caught by these pins.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes
from oracle import closed_shell as cs
from oracle import fci, integrals as ints, solver, spin_orbital as so, thc


def _hamiltonian(o, v, P, G, K, seed, consistent=True):
    s = make_system(o, v, P, G, K, seed, consistent=consistent)
    return s, cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)


def _random_t(o, v, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    t1 = rng.standard_normal((o, v)) * scale
    t2 = rng.standard_normal((o, o, v, v)) * scale
    return t1, 0.5 * (t2 + t2.transpose(1, 0, 3, 2))


def _spin_orbital_residual(s, H, t1, t2):
    g = ints.eri(s.L, s.L)
    f, w = so.spin_blocks(H.h, g, s.o)
    T1, T2 = so.to_spin_amplitudes(t1, t2)
    R1, R2 = so.residual(f, w, T1, T2, 2 * s.o)
    r1, r2 = so.closed_shell_view(R1, R2)
    return r1, r2, so.energy(f, w, T1, T2, 2 * s.o)


@pytest.mark.parametrize("o,v,seed", [(2, 4, 3), (3, 5, 11), (1, 6, 7)])
def test_closed_shell_matches_spin_orbital(o, v, seed):
    s, H = _hamiltonian(o, v, 6, 16, 16, seed)
    t1, t2 = _random_t(o, v, seed + 100)
    r1, r2 = cs.residual(H, t1, t2)
    q1, q2, Eso = _spin_orbital_residual(s, H, t1, t2)
    scale = max(abs(q2).max(), abs(q1).max())
    assert abs(r2 - q2).max() < 1e-12 * scale
    assert abs(r1 - q1).max() < 1e-12 * scale
    assert abs(cs.energy(H, t1, t2) - Eso) < 1e-13


def test_fock_is_canonical_after_backout():
    """h is backed out so that f = diag(eps); the spin-orbital code rebuilds f."""
    s, H = _hamiltonian(3, 5, 6, 16, 16, 2)
    g = ints.eri(s.L, s.L)
    f, _ = so.spin_blocks(H.h, g, s.o)
    ref = np.diag(np.repeat(np.concatenate([s.eps_o, s.eps_v]), 2))
    assert abs(f - ref).max() < 1e-13
    F0 = ints.dressed_fock(H.h, s.L, np.zeros((3, 5)), 3)
    assert abs(F0 - np.diag(np.concatenate([s.eps_o, s.eps_v]))).max() < 1e-13


def test_thc_ovov_equals_cholesky_at_full_rank():
    s, H = _hamiltonian(3, 6, 6, 20, 20, 5)
    assert abs(H.g_ovov_thc - H.g_ovov_chol).max() < 1e-15 * 100


@pytest.mark.parametrize("seed", [0, 1])
def test_two_electron_ccsd_equals_fci(seed):
    s, H = _hamiltonian(1, 7, 8, 30, 30, seed)
    E, t1, t2, _ = solver.solve_canonical(H, s.eps_o, s.eps_v, tol=1e-10)
    g = ints.eri(s.L, s.L)
    E_fci = fci.singlet_ground_energy(H.h, g) - cs.reference_energy(H)
    assert abs(E - E_fci) < 1e-10
    assert abs(E) > 1e-4          # not a trivially uncorrelated system


def test_first_jacobi_step_is_mp2():
    s, H = _hamiltonian(3, 8, 6, 24, 24, 4, consistent=False)
    d1 = s.eps_v[None, :] - s.eps_o[:, None]
    d2 = d1[:, None, :, None] + d1[None, :, None, :]
    r1, r2 = cs.residual(H, np.zeros((3, 8)), np.zeros((3, 3, 8, 8)))
    assert abs(r1).max() < 1e-14          # Brillouin: F_ai = 0
    t2 = -r2 / d2
    E = cs.energy(H, np.zeros((3, 8)), t2)
    assert abs(E - solver.mp2_energy(H, s.eps_o, s.eps_v)) < 1e-14


def test_full_rank_thc_equals_canonical_ccsd():
    o, v = 2, 4
    s, H = _hamiltonian(o, v, o * v, 16, 16, 9)
    E, _, _, _ = solver.solve_canonical(H, s.eps_o, s.eps_v, tol=1e-10)
    Et, Zc, t1, _ = solver.solve_thc(H, s.Y, s.eps_o, s.eps_v, tol=1e-10)
    assert abs(E - Et) < 1e-10
    # RR-MP2 at full rank: one projected Jacobi step from zero is MP2.
    C, e = thc.metric_basis(s.Y, s.eps_o, s.eps_v)
    _, sig = solver.projected_residual(H, s.Y, np.zeros((o * v, o * v)), np.zeros((o, v)))
    T = -(C.T @ sig @ C) / (e[:, None] + e[None, :])
    t2 = thc.amplitudes(s.Y, C @ T @ C.T, o)
    Emp2 = cs.energy(H, np.zeros((o, v)), t2)
    assert abs(Emp2 - solver.mp2_energy(H, s.eps_o, s.eps_v)) < 1e-12


def test_metric_basis_is_semi_unitary_and_diagonalises_fock():
    s, _ = _hamiltonian(3, 7, 12, 20, 20, 1)
    C, e = thc.metric_basis(s.Y, s.eps_o, s.eps_v)
    U = thc.kr(s.Y[:3], s.Y[3:]) @ C
    assert abs(U.T @ U - np.eye(C.shape[1])).max() < 1e-10            # Eq. 12
    d = (s.eps_v[None, :] - s.eps_o[:, None]).ravel()
    assert abs(U.T @ (d[:, None] * U) - np.diag(e)).max() < 1e-10
    assert e.min() >= d.min() - 1e-12 and e.max() <= d.max() + 1e-12


def test_symmetries():
    o, v, P = 3, 6, 10
    s, H = _hamiltonian(o, v, P, 20, 12, 6, consistent=False)
    Zc, t1 = random_amplitudes(P, o, v, 8, t1_scale=0.05)
    t2 = thc.amplitudes(s.Y, Zc, o)
    assert abs(t2 - t2.transpose(1, 0, 3, 2)).max() < 1e-16 * 100
    r1, r2 = cs.residual(H, t1, t2)
    assert abs(r2 - r2.transpose(1, 0, 3, 2)).max() < 1e-13 * abs(r2).max()
    _, sig = solver.projected_residual(H, s.Y, Zc, t1)
    assert abs(sig - sig.T).max() < 1e-13 * abs(sig).max()


def test_projected_residual_is_quadratic_in_core():
    """At fixed t1 the residual is a quadratic polynomial of Zc."""
    o, v, P = 2, 5, 8
    s, H = _hamiltonian(o, v, P, 14, 10, 2, consistent=False)
    Zc, t1 = random_amplitudes(P, o, v, 3, t2_scale=0.05, t1_scale=0.05)
    sig = [solver.projected_residual(H, s.Y, a * Zc, t1)[1] for a in (0, 1, 2, 3)]
    d3 = sig[3] - 3 * sig[2] + 3 * sig[1] - sig[0]
    d2 = sig[2] - 2 * sig[1] + sig[0]
    assert abs(d3).max() < 1e-12 * abs(sig[3]).max()
    assert abs(d2).max() > 1e-6 * abs(sig[3]).max()


def test_residual_is_quartic_in_t1():
    o, v = 2, 4
    s, H = _hamiltonian(o, v, 6, 14, 10, 12, consistent=False)
    t1, t2 = _random_t(o, v, 1, scale=0.2)
    r = [np.concatenate([x.ravel() for x in cs.residual(H, a * t1, t2)])
         for a in range(6)]
    d5 = r[5] - 5 * r[4] + 10 * r[3] - 10 * r[2] + 5 * r[1] - r[0]
    assert abs(d5).max() < 1e-11 * abs(r[5]).max()


def test_gauge_null_space_leaves_residual_unchanged():
    """P > o v: a core change in the null space of y o y changes nothing."""
    o, v, P = 2, 3, 9
    s, H = _hamiltonian(o, v, P, 12, 12, 4, consistent=False)
    Zc, t1 = random_amplitudes(P, o, v, 5, t1_scale=0.05)
    U = thc.kr(s.Y[:o], s.Y[o:])
    _, _, Vt = np.linalg.svd(U)
    n0 = Vt[o * v:].T                         # null space of U, P x (P - ov)
    dZ = n0 @ np.ones((n0.shape[1], n0.shape[1])) @ n0.T
    r1a, sa = solver.projected_residual(H, s.Y, Zc, t1)
    r1b, sb = solver.projected_residual(H, s.Y, Zc + dZ, t1)
    assert abs(sa - sb).max() < 1e-12 * abs(sa).max()
    assert abs(r1a - r1b).max() < 1e-12 * abs(r1a).max()


# ------------------------------------------------------------ planted mistakes

MUTATIONS = {
    "paper_literal_eq35_quarter": ("EQ35_PREFACTOR", 0.25),
    "drop_eq31": ("eq31", lambda D, t2: 0.0 * t2),
    "eq31_undressed": ("eq31", lambda D, t2: _eq31_undressed(D, t2)),
    "eq41_literal_t_ji_ca": ("eq41", lambda H, D, t2: _eq41_literal(H, D, t2)),
    "eq38_transposed_oo": ("eq38", lambda D, t2: _eq38_transposed(D, t2)),
}


def _eq31_undressed(D, t2):
    o = D.o
    L = D._L_undressed
    g = ints.eri(L[:, :o, :o], L[:, o:, o:])     # undressed (kj|bc), [k,j,b,c]
    return (-np.einsum('ikac,kjbc->ijab', t2, g, optimize=True)
            - np.einsum('jkbc,kiac->ijab', t2, g, optimize=True))


def _eq41_literal(H, D, t2):
    """Eq. 41 read literally with (t_ij^ac + t_ji^ca): not pair-symmetric."""
    Fv = D.Fvv() + cs.xi_vv(H, t2)
    Fo = D.Foo() + cs.xi_oo(H, t2)
    tt = t2 + t2.transpose(1, 0, 3, 2)
    return (np.einsum('ijac,bc->ijab', tt, Fv) - np.einsum('ikab,kj->ijab', tt, Fo))


def _eq38_transposed(D, t2):
    """Eq. 38 with the dressed oo block transposed (l_ij for l_ji)."""
    Dt = cs.Dressed.__new__(cs.Dressed)
    Dt.o = D.o
    Dt.F = D.F
    Lh = D.Lh.copy()
    Lh[:, :D.o, :D.o] = Lh[:, :D.o, :D.o].transpose(0, 2, 1)
    Dt.Lh = Lh
    return _orig_eq38(Dt, t2)


_orig_eq38 = cs.eq38


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_are_caught(name, monkeypatch):
    o, v = 2, 4
    s, H = _hamiltonian(o, v, 6, 14, 14, 21)
    t1, t2 = _random_t(o, v, 22)
    q1, q2, _ = _spin_orbital_residual(s, H, t1, t2)
    orig_dressed_init = cs.Dressed.__init__

    def init(self, Hm, t1m):
        orig_dressed_init(self, Hm, t1m)
        self._L_undressed = Hm.L

    monkeypatch.setattr(cs.Dressed, "__init__", init)
    r1, r2 = cs.residual(H, t1, t2)
    assert max(abs(r2 - q2).max(), abs(r1 - q1).max()) < 1e-12   # unmutated
    attr, value = MUTATIONS[name]
    monkeypatch.setattr(cs, attr, value)
    r1, r2 = cs.residual(H, t1, t2)
    err = max(abs(r2 - q2).max(), abs(r1 - q1).max())
    assert err > 1e-6


def test_mp2_density_matches_spin_orbital_and_traces():
    """App. II Eqs. 47-48 against the spin-orbital density summed over spin;
    the two blocks have opposite traces and are symmetric for symmetric t2."""
    from oracle import density, spin_orbital as so
    rng = np.random.default_rng(41)
    o, v = 3, 5
    t2 = rng.standard_normal((o, o, v, v)) * 0.1
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))          # t_ij^ab = t_ji^ba
    Doo, Dvv = density.mp2_density(t2)
    _, T2 = so.to_spin_amplitudes(np.zeros((o, v)), t2)
    Soo, Svv = density.spin_orbital_density(T2, 2 * o)
    assert np.allclose(Doo, Soo[0::2, 0::2] + Soo[1::2, 1::2], atol=1e-14)
    assert np.allclose(Dvv, Svv[0::2, 0::2] + Svv[1::2, 1::2], atol=1e-14)
    assert np.allclose(Doo, Doo.T, atol=1e-14) and np.allclose(Dvv, Dvv.T, atol=1e-14)
    assert abs(np.trace(Doo) + np.trace(Dvv)) < 1e-13


def test_mp2_density_of_a_single_pair_amplitude():
    """Brute force: one non-zero amplitude pair t_00^01 = t_00^10 = s gives
    D_00 = -2 s^2 (2 - 1) * 2 terms and D_vv on the 2 x 2 block."""
    from oracle import density
    o, v, s = 1, 2, 0.3
    t2 = np.zeros((o, o, v, v))
    t2[0, 0, 0, 1] = t2[0, 0, 1, 0] = s
    Doo, Dvv = density.mp2_density(t2)
    # D_00 = -2 sum_ab t^ab (2 t^ab - t^ba) = -2 (s (2s - s) + s (2s - s)) = -4 s^2
    assert Doo[0, 0] == pytest.approx(-4 * s * s)
    # D_ab = 2 sum_c t^ac (2 t^bc - t^bc) = 2 sum_c t^ac t^bc  (i = j = 0)
    assert np.allclose(Dvv, 2 * np.array([[s * s, 0], [0, s * s]]))


def _planted_cp(o, v, N, W, seed):
    rng = np.random.default_rng(seed)
    yo, yv, tau = rng.standard_normal((o, W)), rng.standard_normal((v, W)), rng.standard_normal((N, W))
    U = (yo[:, None, :] * yv[None, :, :]).reshape(o * v, W) @ tau.T
    eps = rng.uniform(0.2, 2.0, N) * rng.choice([-1.0, 1.0], N)
    return U, eps, yo, yv, tau, rng


def test_cp_als_updates_are_exact_minimisers():
    """After each ALS update the gradient of the weighted objective (Eq. 15)
    with respect to the updated factor vanishes (central differences)."""
    from oracle import cp_als
    U, eps, yo, yv, tau, rng = _planted_cp(4, 5, 6, 3, 7)
    U = U + 0.3 * rng.standard_normal(U.shape)          # not exactly low rank
    yo0, yv0, t0 = (a + 0.5 * rng.standard_normal(a.shape) for a in (yo, yv, tau))
    new = cp_als.update_yo(U, eps, yo0, yv0, t0)
    for upd, which in ((new, 0),):
        h = 1e-6
        for idx in np.ndindex(upd.shape):
            d = np.zeros_like(upd); d[idx] = h
            fp = cp_als.objective(U, eps, upd + d, yv0, t0)
            fm = cp_als.objective(U, eps, upd - d, yv0, t0)
            assert abs(fp - fm) / (2 * h) < 1e-6
    nv = cp_als.update_yv(U, eps, new, yv0, t0)
    nt = cp_als.update_tau(U, new, nv)
    h = 1e-6
    for idx in np.ndindex(nv.shape):
        d = np.zeros_like(nv); d[idx] = h
        g = (cp_als.objective(U, eps, new, nv + d, t0) - cp_als.objective(U, eps, new, nv - d, t0)) / (2 * h)
        assert abs(g) < 1e-6
    for idx in np.ndindex(nt.shape):
        d = np.zeros_like(nt); d[idx] = h
        g = (cp_als.objective(U, eps, new, nv, nt + d) - cp_als.objective(U, eps, new, nv, nt - d)) / (2 * h)
        assert abs(g) < 1e-6


def test_cp_als_recovers_a_planted_factorisation_monotonically():
    from oracle import cp_als
    U, eps, yo, yv, tau, rng = _planted_cp(6, 8, 7, 4, 11)
    start = [a + 0.1 * rng.standard_normal(a.shape) for a in (yo, yv, tau)]
    _, _, _, hist = cp_als.als(U, eps, *start, 60)
    assert all(b <= a * (1 + 1e-12) + 1e-300 for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 1e-16 * max(1.0, float(np.sum(U ** 2)))
