"""Full-size (o=40, v=200, P=400, G=1200, K=600) checks of the CUDA path.

The oracle cannot form every 4-index piece at this size (the vvvv block alone
is 12.8 GB), so the full residual is checked through what the oracle can
still compute exactly and through properties that hold at any size:
  * Zc = 0, t1 != 0: sigma is the projection of the dressed (ai^|bj) and
    Omega_i^a = F^_ai, both formed plainly by the oracle;
  * the CCSD energy at a random (Zc, t1), formed plainly by the oracle;
  * sigma is symmetric and exactly quadratic in Zc at fixed t1.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes, CONFIGS
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["fp64", "fp64tc"])
def o40_system(request):
    """The bench system in a float64 context: CUDA-core products, and the
    tensor-core integer-slice products the benchmark runs by default."""
    import __graft_entry__ as g
    g.build()
    import paper_2111_11473_gb300 as pkg
    o, v, P, G, K, seed = CONFIGS["o40_v200_P400_G1200_K600"]
    s = make_system(o, v, P, G, K, seed)
    from oracle import closed_shell as cs
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    prec = {"fp64": pkg.THC_PREC_FP64, "fp64tc": pkg.THC_PREC_FP64_TC}[request.param]
    ctx = context(s, precision=prec)
    yield s, H, ctx
    ctx.close()


def test_fullsize_singles_only_state(o40_system):
    s, H, ctx = o40_system
    from oracle import closed_shell as cs, thc
    _, t1 = random_amplitudes(s.P, s.o, s.v, 77, t1_scale=0.02)
    Zc = np.zeros((s.P, s.P))
    sig, sig1, E = ctx.residual(Zc, t1)
    D = cs.Dressed(H, t1)
    g_vovo = D.g('vovo').transpose(1, 3, 0, 2)          # [i, j, a, b] = (ai^|bj)
    sig_ref = thc.project(s.Y, g_vovo, s.o)
    r1_ref = D.Fvo().T
    assert np.abs(sig - sig_ref).max() < 1e-10
    assert np.abs(sig1 - r1_ref).max() < 1e-10
    assert abs(E - cs.energy(H, t1, np.zeros((s.o, s.o, s.v, s.v)))) < 1e-9


def test_fullsize_energy_and_structure(o40_system):
    s, H, ctx = o40_system
    from oracle import closed_shell as cs, thc
    Zc, t1 = random_amplitudes(s.P, s.o, s.v, 78, t2_scale=0.01, t1_scale=0.01)
    sig = []
    for a in (0.0, 1.0, 2.0, 3.0):
        r, r1, E = ctx.residual(a * Zc, t1)
        sig.append(r)
        if a == 1.0:
            E1 = E
            assert np.abs(r - r.T).max() < 1e-12 * np.abs(r).max()
    E_ref = cs.energy(H, t1, thc.amplitudes(s.Y, Zc, s.o))
    assert abs(E1 - E_ref) < 1e-9
    d3 = sig[3] - 3 * sig[2] + 3 * sig[1] - sig[0]
    d2 = sig[2] - 2 * sig[1] + sig[0]
    assert np.abs(d3).max() < 1e-9 * np.abs(sig[3]).max()
    assert np.abs(d2).max() > 1e-6 * np.abs(sig[3]).max()
