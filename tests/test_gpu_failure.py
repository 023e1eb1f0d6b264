"""Failure detection on the GPU without a fault: bounded device waits.

Every waiting kernel of the library (TMA/MMA pipelines, the triangle
kernel's operand ring) spins on an mbarrier with a clock budget; on expiry
it raises a device flag, drains what it issued and returns, and the host
reports THC_ERR_TIMEOUT.  thc_selftest_bounded_wait runs that path on a
barrier nothing completes (about 1 ms budget); the device must stay usable.
"""
import numpy as np
import pytest

from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def test_expired_wait_is_reported_and_device_stays_usable():
    import paper_2111_11473_gb300 as pkg
    from paper_2111_11473_gb300 import binding
    assert binding.selftest_bounded_wait(True) == "THC_OK"
    assert binding.selftest_bounded_wait(False) == "THC_ERR_TIMEOUT"
    assert "expired" in pkg.load_library().thc_last_error(None).decode()
    # the device still computes correctly after the expired wait
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(3, 7, 10, 14, 9, 5)
    with context(s) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < 1e-10
    assert abs(E - E_ref) < 1e-9
    assert binding.selftest_bounded_wait(True) == "THC_OK"


@pytest.mark.parametrize("seed", [1, 2])
def test_tensor_core_product_randomised(seed):
    """tcgen05 bf16 hi/lo products against the CUDA-core products over random
    shapes, orientations, batch modes, split-K and beta (64 cases a seed)."""
    from paper_2111_11473_gb300 import binding
    status, max_rel, failures = binding.selftest_gemm(cases=64, seed=seed)
    print(f"\nseed {seed}: max bf16x3 relative difference {max_rel:.2e}, failures {failures}")
    assert status == "THC_OK" and failures == 0
    assert max_rel < 1e-3
