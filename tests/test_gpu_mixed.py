"""Mixed-precision path: float32 storage, tensor-core products with bf16
hi/lo splitting (or float32 CUDA cores), float32 triangle kernel, float64
accumulation of sigma and of the energy.

Bounds relative to the largest |sigma| entry, from the arithmetic of each
policy (inner lengths up to 25600 here):
  tc_products = 0  float32 FMA chains: 2e-5
  tc_products = 3  bf16 hi*hi + hi*lo + lo*hi: each product is off by at most
                   about 3 * 2^-17 (the dropped lo*lo term and the two split
                   roundings), float32 accumulation: 1e-4
  tc_products = 1  bf16 hi*hi only: 2^-8 per factor: 3e-2
The energy is accumulated in float64 from float32 weights: 1e-6 relative.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes, CONFIGS
from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu

BOUND = {0: 2e-5, 3: 1e-4, 1: 3e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


CASES = [(3, 7, 10, 14, 9, 5), (7, 37, 70, 90, 45, 11), (5, 20, 60, 120, 60, 0),
         (8, 60, 120, 200, 80, 13)]


@pytest.mark.parametrize("tcp", [3, 0, 1])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_mixed_matches_oracle_within_bound(case, tcp):
    import paper_2111_11473_gb300 as pkg
    o, v, P, G, K, seed = case
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(o, v, P, G, K, seed)
    with context(s, precision=pkg.THC_PREC_MIXED, tc_products=tcp) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    scale = max(np.abs(sig_ref).max(), np.abs(r1_ref).max())
    err = max(np.abs(sig - sig_ref).max(), np.abs(sig1 - r1_ref).max())
    print(f"mixed tc={tcp} {case}: max|d sigma| / max|sigma| = {err / scale:.2e}, "
          f"|dE| = {abs(E - E_ref):.2e}")
    assert err < BOUND[tcp] * scale
    assert abs(E - E_ref) < 1e-6 * max(1e-3, abs(E_ref))


@pytest.mark.parametrize("route", [1, 2])
def test_mixed_alg7_routes(route):
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(8, 60, 120, 200, 80, 13)
    with context(s, precision=pkg.THC_PREC_MIXED, alg7_route=route) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    scale = max(np.abs(sig_ref).max(), np.abs(r1_ref).max())
    err = max(np.abs(sig - sig_ref).max(), np.abs(sig1 - r1_ref).max())
    print(f"mixed alg7 route {route}: {err / scale:.2e}")
    assert err < BOUND[3] * scale


@pytest.mark.parametrize("tcp", [3, 0])
def test_mixed_fullsize_error_against_fp64_gpu(tcp):
    import paper_2111_11473_gb300 as pkg
    o, v, P, G, K, seed = CONFIGS["o40_v200_P400_G1200_K600"]
    s = make_system(o, v, P, G, K, seed)
    Zc, t1 = random_amplitudes(P, o, v, 78, t2_scale=0.01, t1_scale=0.01)
    with context(s) as c64:
        sig64, s164, E64 = c64.residual(Zc, t1)
    with context(s, precision=pkg.THC_PREC_MIXED, tc_products=tcp) as c32:
        sig32, s132, E32 = c32.residual(Zc, t1)
    scale = max(np.abs(sig64).max(), np.abs(s164).max())
    err = max(np.abs(sig32 - sig64).max(), np.abs(s132 - s164).max())
    print(f"mixed tc={tcp} vs fp64 at full size: rel {err / scale:.2e}, "
          f"|dE| = {abs(E32 - E64):.2e} Eh")
    assert err < BOUND[tcp] * scale
    assert abs(E32 - E64) < 1e-6 * abs(E64)


@pytest.mark.parametrize("route", [1, 2])
def test_mixed_t2sq_routes_within_bound(route):
    """Alg. 6 (triangle) and Algs. 4-5 (tensor-core products) in mixed precision."""
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(8, 60, 120, 200, 80, 13)
    with context(s, precision=pkg.THC_PREC_MIXED, t2sq_route=route) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    scale = max(np.abs(sig_ref).max(), np.abs(r1_ref).max())
    err = max(np.abs(sig - sig_ref).max(), np.abs(sig1 - r1_ref).max())
    assert err < BOUND[3] * scale
    assert abs(E - E_ref) < 1e-6 * max(1e-3, abs(E_ref))


def test_mixed_mp2_density_within_bound():
    """App. II density matrices on the tensor cores (bf16x3) against Eqs. 47-48."""
    import paper_2111_11473_gb300 as pkg
    from oracle import density, thc
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(8, 60, 120, 200, 80, 13)
    Doo_ref, Dvv_ref = density.mp2_density(thc.amplitudes(s.Y, Zc, 8))
    with context(s, precision=pkg.THC_PREC_MIXED) as ctx:
        Doo, Dvv = ctx.mp2_density(Zc)
    scale = max(np.abs(Doo_ref).max(), np.abs(Dvv_ref).max())
    assert np.abs(Doo - Doo_ref).max() < BOUND[3] * scale
    assert np.abs(Dvv - Dvv_ref).max() < BOUND[3] * scale
