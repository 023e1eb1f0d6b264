"""Mixed-precision path (float32 storage, split-bf16 tensor-core products,
float32 triangle kernel, float64 accumulation of sigma and the energy).

Bound: every contraction accumulates in float32, so each output carries a
relative error of a few units of 2^-24 times the square root of its inner
length, times the condition of the sum; 2e-5 of the largest |sigma| entry
covers the inner lengths here (<= 1200) with margin.  The energy is
accumulated in float64, but its weights are float32 products (inner length
o, about sqrt(o) 2^-24 each): 1e-6 relative.
"""
import numpy as np
import pytest

from synth import make_system, random_amplitudes, CONFIGS
from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu

REL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("case", [(3, 7, 10, 14, 9, 5), (7, 37, 70, 90, 45, 11),
                                  (5, 20, 60, 120, 60, 0)], ids=lambda c: "x".join(map(str, c)))
def test_mixed_matches_oracle_within_float32_bound(case):
    import paper_2111_11473_gb300 as pkg
    o, v, P, G, K, seed = case
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(o, v, P, G, K, seed)
    with context(s, precision=pkg.THC_PREC_MIXED) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    scale = max(np.abs(sig_ref).max(), np.abs(r1_ref).max())
    err = max(np.abs(sig - sig_ref).max(), np.abs(sig1 - r1_ref).max())
    print(f"mixed {case}: max|d sigma| / max|sigma| = {err / scale:.2e}, |dE| = {abs(E - E_ref):.2e}")
    assert err < REL * scale
    assert abs(E - E_ref) < 1e-6 * max(1e-3, abs(E_ref))


def test_mixed_fullsize_error_against_fp64_gpu():
    import paper_2111_11473_gb300 as pkg
    o, v, P, G, K, seed = CONFIGS["c2"]
    s = make_system(o, v, P, G, K, seed)
    Zc, t1 = random_amplitudes(P, o, v, 78, t2_scale=0.01, t1_scale=0.01)
    with context(s) as c64:
        sig64, s164, E64 = c64.residual(Zc, t1)
    with context(s, precision=pkg.THC_PREC_MIXED) as c32:
        sig32, s132, E32 = c32.residual(Zc, t1)
    scale = max(np.abs(sig64).max(), np.abs(s164).max())
    err = max(np.abs(sig32 - sig64).max(), np.abs(s132 - s164).max())
    print(f"mixed vs fp64 at full size: rel {err / scale:.2e}, |dE| = {abs(E32 - E64):.2e} Eh")
    assert err < REL * scale
    assert abs(E32 - E64) < 1e-6 * abs(E64)
