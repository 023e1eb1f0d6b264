"""Float64 products on the tensor cores (THC_PREC_FP64_TC): exact integer
slices, float64 combination.  Held to the float64 bars (needs a GB300):
residual max-abs 1e-10 and energy 1e-9 Eh against the oracle, and agreement
with the float64 CUDA-core path to float64 rounding."""
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


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_selftest_against_cuda_core_products(seed):
    """Random shapes, orientations, batch modes, beta, up to three exact K
    chunks, entries spread over 2^-40 .. 1."""
    import paper_2111_11473_gb300 as pkg
    status, max_rel, failures = pkg.binding.selftest_gemm_f64(cases=48, seed=seed)
    print(f"seed {seed}: max relative difference {max_rel:.2e}")
    assert status == "THC_OK" and failures == 0
    assert max_rel < 1e-13


CASES = [(3, 7, 10, 14, 9, 5), (7, 37, 70, 90, 45, 11), (5, 20, 60, 120, 60, 0),
         (8, 60, 120, 200, 80, 13), (1, 9, 12, 20, 7, 3)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c)))
def test_residual_matches_oracle(case):
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(*case)
    with context(s, precision=pkg.THC_PREC_FP64_TC) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert np.abs(sig1 - r1_ref).max() < RES_TOL
    assert abs(E - E_ref) < E_TOL


@pytest.mark.parametrize("kw", [dict(alg7_route=1), dict(alg7_route=2), dict(x_block6=32),
                                dict(x_block6=31, i_chunk=37),
                                dict(k_slab=7, i_chunk=13, x_block=5), dict(t2sq_route=2)],
                         ids=["alg7_blocked", "alg7_dense", "x6_32", "x6_31_odd",
                              "small_blocks", "algs45"])
def test_routes_and_blocking_match_cuda_core_float64(kw):
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(8, 60, 120, 200, 80, 13)
    with context(s, precision=pkg.THC_PREC_FP64_TC, **kw) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    with context(s, precision=pkg.THC_PREC_FP64, **kw) as ctx:
        sig0, sig10, E0 = ctx.residual(Zc, t1)
    scale = max(np.abs(sig0).max(), np.abs(sig10).max())
    d = max(np.abs(sig - sig0).max(), np.abs(sig1 - sig10).max())
    print(f"{kw}: max |tc - cuda cores| / max |sigma| = {d / scale:.2e}")
    assert d < 1e-12 * scale
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert abs(E - E_ref) < E_TOL


def test_fullsize_agrees_with_cuda_core_float64():
    """o=40, v=200, P=400, G=1200, K=600 at the bench state."""
    import paper_2111_11473_gb300 as pkg
    from synth import CONFIGS, make_system
    o, v, P, G, K, seed = CONFIGS["o40_v200_P400_G1200_K600"]
    s = make_system(o, v, P, G, K, seed)
    with context(s) as ctx:
        Zc, t1, _ = ctx.solve(max_iter=3, diis_n=0, raise_on_failure=False)
        sig0, sig10, E0 = ctx.residual(Zc, t1)
    with context(s, precision=pkg.THC_PREC_FP64_TC) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    scale = max(np.abs(sig0).max(), np.abs(sig10).max())
    d = max(np.abs(sig - sig0).max(), np.abs(sig1 - sig10).max())
    print(f"o=40: max |tc - cuda cores| = {d:.2e} (max |sigma| {scale:.2e}), dE = {E - E0:.2e}")
    # sigma (5e-5 here) is a sum of terms of order 1: both paths carry
    # float64 rounding of those terms
    assert d < 1e-14
    assert abs(E - E0) < 1e-12


def test_solve_converges_to_the_float64_energy():
    import paper_2111_11473_gb300 as pkg
    s, *_ = oracle_case(5, 20, 60, 120, 60, 0)
    with context(s) as ctx:
        _, _, r0 = ctx.solve(r_tol=1e-9, max_iter=60)
    with context(s, precision=pkg.THC_PREC_FP64_TC) as ctx:
        _, _, r1 = ctx.solve(r_tol=1e-9, max_iter=60)
    assert r1.status == "THC_OK"
    assert abs(r1.energy - r0.energy) < 1e-11
