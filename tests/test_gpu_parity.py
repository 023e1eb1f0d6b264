"""CUDA path vs the FP64 oracle, element by element (needs a GB300).

Tolerances: residual max-abs 1e-10 and energy 1e-9 Eh in FP64.
"""
import numpy as np
import pytest

from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu

RES_TOL = 1e-10
E_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


CASES = [
    # o, v, P, G, K, seed: tiny; several 64-tiles with ragged tails; the o=5, v=20, P=60 shape
    (3, 7, 10, 14, 9, 5),
    (7, 37, 70, 90, 45, 11),
    (5, 20, 60, 120, 60, 0),
    (1, 9, 12, 20, 7, 3),          # one occupied orbital
    (4, 5, 1, 6, 3, 8),            # rank-one amplitudes
    (2, 6, 9, 1, 1, 4),            # one grid point, one Cholesky vector
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_residual_matches_oracle(case):
    o, v, P, G, K, seed = case
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(o, v, P, G, K, seed)
    with context(s) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert np.abs(sig1 - r1_ref).max() < RES_TOL
    assert abs(E - E_ref) < E_TOL
    assert np.abs(sig - sig.T).max() < 1e-12 * max(1.0, np.abs(sig).max())


def test_blocking_partition_invariance():
    """Any split into Cholesky slabs, grid chunks and X blocks gives the same result."""
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(7, 37, 70, 90, 45, 11)
    results = []
    for kb, ic, xb in [(0, 0, 0), (7, 13, 5), (45, 90, 70), (1, 1, 1)]:
        with context(s, k_slab=kb, i_chunk=ic, x_block=xb) as ctx:
            results.append(ctx.residual(Zc, t1))
    for sig, sig1, E in results:
        assert np.abs(sig - sig_ref).max() < RES_TOL
        assert np.abs(sig1 - r1_ref).max() < RES_TOL
        assert abs(E - E_ref) < E_TOL
    for sig, sig1, E in results[1:]:
        assert np.abs(sig - results[0][0]).max() < 1e-12


def test_zero_amplitudes_give_bare_integrals_and_mp2():
    """At Zc = 0, t1 = 0 the residual is the projected (ai|bj); energy is zero."""
    s, _, _, _, _, _ = oracle_case(4, 11, 16, 30, 20, 2)
    Zc = np.zeros((16, 16))
    t1 = np.zeros((4, 11))
    from oracle import closed_shell as cs, solver as osolver
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    r1, sg = osolver.projected_residual(H, s.Y, Zc, t1)
    with context(s) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
        assert ctx.energy(Zc, t1) == 0.0
    assert np.abs(sig - sg).max() < RES_TOL
    assert np.abs(sig1).max() < RES_TOL        # Brillouin: F_ai = 0
    assert E == 0.0


def test_device_pointers_and_energy_entry_point():
    torch = pytest.importorskip("torch")
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(3, 7, 10, 14, 9, 5)
    dev = torch.device("cuda:0")
    tens = [torch.from_numpy(a).to(dev) for a in (s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z)]
    import paper_2111_11473_gb300 as pkg
    with pkg.Context(*tens, stream=torch.cuda.current_stream()) as ctx:
        sig, sig1, E = ctx.residual(torch.from_numpy(Zc).to(dev), torch.from_numpy(t1).to(dev))
        assert sig.is_cuda and sig1.is_cuda
        assert (sig.cpu().numpy() - sig_ref).__abs__().max() < RES_TOL
        assert (sig1.cpu().numpy() - r1_ref).__abs__().max() < RES_TOL
        assert abs(E - E_ref) < E_TOL
        assert abs(ctx.energy(Zc, t1) - E_ref) < E_TOL


def test_argument_and_numeric_errors():
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, *_ = oracle_case(3, 7, 10, 14, 9, 5)
    with context(s) as ctx:
        bad = Zc.copy()
        bad[0, 1] += 1.0
        with pytest.raises(pkg.ThcError) as e:
            ctx.residual(bad, t1)
        assert e.value.name == "THC_ERR_ARG"
        t1n = t1.copy()
        t1n[0, 0] = np.nan
        with pytest.raises(pkg.ThcError) as e:
            ctx.residual(Zc, t1n)
        assert e.value.name == "THC_ERR_NUMERIC"
        # the context stays usable after an error
        sig, _, _ = ctx.residual(Zc, t1)
        assert np.isfinite(sig).all()
    zbad = s.z.copy()
    zbad[0, 1] += 1.0
    with pytest.raises(pkg.ThcError) as e:
        pkg.Context(s.eps_o, s.eps_v, s.Y, s.L, s.x, zbad)
    assert e.value.name == "THC_ERR_ARG"


@pytest.mark.parametrize("route", [1, 2])
def test_alg7_routes_match_oracle(route):
    """Alg. 7 through the THC factors (as printed) and through the dense (ib|ja)."""
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(7, 37, 70, 90, 45, 11)
    with context(s, alg7_route=route, x_block=9) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert np.abs(sig1 - r1_ref).max() < RES_TOL


@pytest.mark.parametrize("case", [(3, 7, 10, 14, 9, 5), (7, 37, 70, 90, 45, 11)],
                         ids=lambda c: "x".join(map(str, c)))
def test_t2sq_n5_route_matches_oracle(case):
    """Eqs. 32-33 through Algs. 4 and 5 (O(N^5), batched products) instead of Alg. 6."""
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(*case)
    with context(s, t2sq_route=2) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert np.abs(sig1 - r1_ref).max() < RES_TOL
    assert abs(E - E_ref) < 1e-9


@pytest.mark.parametrize("case", [(3, 7, 10, 14, 9, 5), (7, 37, 70, 90, 45, 11)],
                         ids=lambda c: "x".join(map(str, c)))
def test_mp2_density_matches_oracle(case):
    """App. II: THC-factorised density matrices (Eqs. 49-56) against Eqs. 47-48."""
    from oracle import density, thc
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(*case)
    Doo_ref, Dvv_ref = density.mp2_density(thc.amplitudes(s.Y, Zc, case[0]))
    with context(s) as ctx:
        Doo, Dvv = ctx.mp2_density(Zc)
    scale = max(np.abs(Doo_ref).max(), np.abs(Dvv_ref).max())
    assert np.abs(Doo - Doo_ref).max() < 1e-12 * max(1.0, scale)
    assert np.abs(Dvv - Dvv_ref).max() < 1e-12 * max(1.0, scale)
