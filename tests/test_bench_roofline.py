"""The triangle roofline that bench.py reports (no GPU needed): the counts
per term each triangle kernel issues, and the fractions derived from them."""
import importlib
import math

import pytest


@pytest.fixture()
def bench():
    b = importlib.import_module("bench")
    b.set_workload("o40_v200_P400_G1200_K600")
    yield b
    b.set_workload(b.DEFAULT_WORKLOAD)


def _terms(w):
    return w["G"] * w["P"] ** 3


def test_mixed_roofline_counts_two_lane_operations_per_term(bench):
    w = bench.WORKLOAD
    flops = 5.0 * _terms(w)          # one residual, one launch
    ms = 8.54
    r = bench.triangle_roofline("mixed", flops, ms, 1, 0.47)
    assert r["kernel"].startswith("k_triangle_pair")
    achieved = flops / (ms * 1e-3) / 1e12
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-12)
    # 80.55 TFLOP/s FP32 peak: the pipe runs 40.27e12 lane operations / s
    pipe = bench.FP32_ALU_TFLOPS * 1e12 / 2.0
    assert math.isclose(r["frac_issued"], achieved * 1e12 / 5.0 * 2.0 / pipe, rel_tol=1e-12)
    assert math.isclose(r["frac"], achieved / bench.FP32_ALU_TFLOPS, rel_tol=1e-12)
    assert r["traffic"] == pytest.approx(12.702e9 + 0.249e9)


def test_unpaired_float32_kernel_for_p_not_a_multiple_of_four(bench, monkeypatch):
    w = dict(bench.WORKLOAD)
    w["P"] = 70
    monkeypatch.setattr(bench, "WORKLOAD", w)
    flops = 5.0 * _terms(w)
    r = bench.triangle_roofline("mixed", flops, 1.0, 1, 0.5)
    assert r["kernel"].startswith("k_triangle_f32")
    pipe = bench.FP32_ALU_TFLOPS * 1e12 / 2.0
    assert math.isclose(r["frac_issued"], r["achieved"] * 1e12 / 5.0 * 3.0 / pipe,
                        rel_tol=1e-12)


def test_float_pair_kernel_is_measured_against_its_own_bound(bench):
    w = bench.WORKLOAD
    flops = 5.0 * _terms(w)
    ms = 68.7
    r = bench.triangle_roofline("fp64tc", flops, ms, 1, 0.5)
    assert r["kernel"].startswith("k_triangle_df")
    # the bound: the FP32 pipe's lane rate / 21.5 operations per term, 5 flops each
    bound = bench.FP32_ALU_TFLOPS / 2.0 / 21.5 * 5.0
    assert math.isclose(r["peak"], bound, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["achieved"] / bound, rel_tol=1e-12)
    assert r["frac"] == pytest.approx(r["frac_issued"], rel=1e-12)
    assert r["frac_of_fp64_alu_peak"] > 4.0        # 5.59 TFLOP/s against 1.26


def test_float64_kernel_fraction_of_the_fp64_peak(bench):
    w = bench.WORKLOAD
    flops = 5.0 * _terms(w)
    r = bench.triangle_roofline("fp64", flops, 301.0, 1, 0.37)
    assert r["kernel"].startswith("k_triangle_sym64")
    assert math.isclose(r["frac"], r["achieved"] / bench.FP64_ALU_TFLOPS, rel_tol=1e-12)
    # it issues 3.5 float64 flops per term, fewer than the 5 counted
    assert r["frac_issued"] == pytest.approx(r["frac"] * 3.5 / 5.0, rel=1e-12)
