"""Per-step arithmetic policy (thc_config.policy) against the oracle and
against the uniform policies (needs a GB300).

  * a policy outside the context's family is rejected (THC_ERR_ARG);
  * naming the context's own policy for every step changes nothing;
  * a float64 tensor-core context whose triangle runs in native float64
    agrees with the CUDA-core float64 path to float64 rounding, and the
    float-pair triangle alone stays within 1e-10 of the oracle;
  * a mixed context with bf16x1 products in one step and bf16x3 elsewhere
    stays within the bf16x1 bound (3e-2 of max|sigma|) and, for the T2^2
    steps whose terms are quadratic in small amplitudes, much closer.
"""
import numpy as np
import pytest

from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu

CASE = (8, 60, 120, 200, 80, 13)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def case():
    return oracle_case(*CASE)


def _err(out, ref):
    sig, sig1, E = out
    _, _, _, sig_ref, r1_ref, E_ref = ref
    scale = max(np.abs(sig_ref).max(), np.abs(r1_ref).max())
    return max(np.abs(sig - sig_ref).max(), np.abs(sig1 - r1_ref).max()), scale, abs(E - E_ref)


def test_policy_outside_the_family_is_rejected(case):
    import paper_2111_11473_gb300 as pkg
    s = case[0]
    with pytest.raises(pkg.ThcError) as e:
        context(s, precision=pkg.THC_PREC_FP64, policy={"alg1": "bf16"})
    assert "policy of step alg1" in str(e.value)
    with pytest.raises(pkg.ThcError):
        context(s, precision=pkg.THC_PREC_MIXED, policy={"triangle": "bf16x3"})
    with pytest.raises(pkg.ThcError):
        context(s, precision=pkg.THC_PREC_MIXED, policy={"alg7": "fp64tc"})


@pytest.mark.parametrize("prec,name", [("fp64", "fp64"), ("fp64tc", "fp64tc"),
                                       ("mixed", "bf16x3")])
def test_explicit_default_policy_is_identical(case, prec, name):
    import paper_2111_11473_gb300 as pkg
    from paper_2111_11473_gb300.binding import STEPS
    s, Zc, t1 = case[:3]
    p = {"fp64": pkg.THC_PREC_FP64, "fp64tc": pkg.THC_PREC_FP64_TC,
         "mixed": pkg.THC_PREC_MIXED}[prec]
    pol = {st: name for st in STEPS}
    if prec == "mixed":
        pol["triangle"] = "fp32"
    with context(s, precision=p) as c:
        a = c.residual(Zc, t1)
    with context(s, precision=p, policy=pol) as c:
        b = c.residual(Zc, t1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_fp64tc_with_native_triangle_matches_cuda_core_float64(case):
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1 = case[:3]
    with context(s, precision=pkg.THC_PREC_FP64) as c:
        ref = c.residual(Zc, t1)
    with context(s, precision=pkg.THC_PREC_FP64_TC, policy={"triangle": "fp64"}) as c:
        out = c.residual(Zc, t1)
    scale = max(np.abs(ref[0]).max(), np.abs(ref[1]).max())
    d = max(np.abs(out[0] - ref[0]).max(), np.abs(out[1] - ref[1]).max())
    print(f"tensor-core products, float64 triangle vs CUDA cores: {d / scale:.2e}")
    assert d < 1e-12 * scale
    err, scale, dE = _err(out, case)
    assert err < 1e-10 and dE < 1e-9


def test_float_pair_triangle_alone(case):
    """Float64 CUDA-core products with only the triangle in float pairs."""
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1 = case[:3]
    with context(s, precision=pkg.THC_PREC_FP64, policy={"triangle": "fp64tc"}) as c:
        out = c.residual(Zc, t1)
    err, scale, dE = _err(out, case)
    print(f"float-pair triangle: max|d| {err:.2e} ({err / scale:.2e} of max|sigma|), dE {dE:.2e}")
    assert err < 1e-10 and dE < 1e-9


@pytest.mark.parametrize("step", ["alg1", "alg2_8", "alg6_gemm", "alg7", "fock"])
def test_mixed_one_step_bf16(case, step):
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1 = case[:3]
    with context(s, precision=pkg.THC_PREC_MIXED, policy={step: "bf16"}) as c:
        out = c.residual(Zc, t1)
    err, scale, dE = _err(out, case)
    print(f"bf16 in {step}: {err / scale:.2e} of max|sigma|, dE {dE:.2e}")
    assert err < 3e-2 * scale
