"""Host-side helpers of the solve comparisons (no GPU needed)."""
from paper_2111_11473_gb300 import precond


def test_time_to_reports_the_first_iteration_within_tolerance():
    hist = [(-0.0030, 1e-2, 0.1), (-0.0040, 1e-3, 0.2), (-0.0041105, 1e-4, 0.3),
            (-0.0041110, 1e-5, 0.4), (-0.0041112, 1e-6, 0.5)]
    # |E - ref| < 1e-6 first at the third entry (5e-7 away)
    assert precond.time_to(hist, -0.0041110, 1e-6) == (3, 0.3)
    assert precond.time_to(hist, -0.0041110, 1e-8) == (4, 0.4)
    assert precond.time_to(hist, -1.0, 1e-6) == (None, None)
    assert precond.time_to([], -0.0041110) == (None, None)


def test_family_sizes_keep_the_bench_ratios():
    # v = 5o, P = 10o, G = 30o, K = 15o: o=40 gives the o=40 bench system's shape
    assert precond.family_sizes(40) == (40, 200, 400, 1200, 600)
    assert precond.family_sizes(60) == (60, 300, 600, 1800, 900)
