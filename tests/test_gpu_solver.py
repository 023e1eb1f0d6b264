"""thc_solve (Jacobi + DIIS on the GPU) against the oracle's solvers."""
import numpy as np
import pytest

from synth import make_system
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_converged_energy_matches_oracle_solver():
    from oracle import closed_shell as cs, solver as osolver
    s = make_system(5, 20, 60, 120, 60, 0)
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    E_ref, Zc_ref, t1_ref, _ = osolver.solve_thc(H, s.Y, s.eps_o, s.eps_v, tol=1e-9)
    with context(s) as ctx:
        Zc, t1, rep = ctx.solve(r_tol=1e-9)
        assert rep.status == "THC_OK" and rep.r_norm < 1e-9
        assert abs(rep.energy - E_ref) < 1e-9
        # the returned point is a zero of the projected residual
        sig, sig1, E = ctx.residual(Zc, t1)
        assert abs(E - rep.energy) < 1e-12
        r1, sg = osolver.projected_residual(H, s.Y, Zc, t1)
        assert np.abs(sg).max() < 1e-8 and np.abs(r1).max() < 1e-8
    assert np.abs(t1 - t1_ref).max() < 1e-7


def test_full_rank_solve_equals_canonical_ccsd():
    from oracle import closed_shell as cs, solver as osolver
    s = make_system(2, 4, 8, 16, 16, 9, consistent=True)
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    E_ref, *_ = osolver.solve_canonical(H, s.eps_o, s.eps_v, tol=1e-11)
    with context(s) as ctx:
        _, _, rep = ctx.solve(r_tol=1e-11)
    assert abs(rep.energy - E_ref) < 1e-10


def test_two_electron_solve_equals_fci():
    from oracle import closed_shell as cs, fci, integrals as ints
    s = make_system(1, 7, 7, 30, 30, 0, consistent=True)
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    E_fci = fci.singlet_ground_energy(H.h, ints.eri(s.L, s.L)) - cs.reference_energy(H)
    with context(s) as ctx:
        _, _, rep = ctx.solve(r_tol=1e-11)
    assert abs(rep.energy - E_fci) < 1e-10


def test_iteration_cap_reports_not_converged():
    import paper_2111_11473_gb300 as pkg
    s = make_system(5, 20, 60, 120, 60, 0)
    with context(s) as ctx:
        Zc, t1, rep = ctx.solve(r_tol=1e-14, max_iter=3, raise_on_failure=False)
        assert rep.status == "THC_ERR_NOT_CONVERGED" and rep.iters == 3
        with pytest.raises(pkg.ThcError):
            ctx.solve(r_tol=1e-14, max_iter=2)
