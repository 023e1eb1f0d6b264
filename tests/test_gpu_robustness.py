"""Failure injection, NaN-poisoned workspaces and checkpoint/resume of the
solver (needs a GB300; nothing here faults, traps or hangs the GPU: the
failures are injected on the host)."""
import os

import numpy as np
import pytest

from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture
def env():
    """Set environment variables for the library's next thc_init calls."""
    saved = {}

    def put(name, value):
        saved.setdefault(name, os.environ.get(name))
        os.environ[name] = value
    yield put
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_injected_allocation_failures_are_clean(prec, env):
    """The n-th device allocation of thc_init fails: every n gives
    THC_ERR_OOM (or, past the last allocation, a working context), and no
    device memory is left behind."""
    torch = pytest.importorskip("torch")
    import paper_2111_11473_gb300 as pkg
    p = {"fp64": pkg.THC_PREC_FP64, "mixed": pkg.THC_PREC_MIXED}[prec]
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(7, 37, 70, 90, 45, 11)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for n in (1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233):
        env("THC_FAIL_ALLOC_AT", str(n))
        try:
            ctx = context(s, precision=p)
        except pkg.ThcError as e:
            assert e.name == "THC_ERR_OOM", str(e)
            assert "injected" in str(e)
            failed += 1
            continue
        with ctx:
            sig, sig1, E = ctx.residual(Zc, t1)
        tol = 1e-10 if prec == "fp64" else 1e-4 * np.abs(sig_ref).max()
        assert np.abs(sig - sig_ref).max() < tol
    assert failed >= 8
    env("THC_FAIL_ALLOC_AT", "0")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (256 << 20)
    with context(s, precision=p) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    tol = 1e-10 if prec == "fp64" else 1e-4 * np.abs(sig_ref).max()
    assert np.abs(sig - sig_ref).max() < tol


CONFIGS = [dict(), dict(alg7_route=1), dict(x_block6=32, i_chunk=13, k_slab=7),
           dict(t2sq_route=2)]


@pytest.mark.parametrize("prec", ["fp64", "fp64tc", "mixed"])
@pytest.mark.parametrize("kw", CONFIGS, ids=["auto", "alg7_blocked", "small_blocks", "algs45"])
def test_poisoned_workspaces_give_identical_results(prec, kw, env):
    """Every scratch buffer filled with NaN bytes at init: the residual, the
    energy and a short solve are bit-identical to an unpoisoned context, so
    no step reads scratch it has not written."""
    import paper_2111_11473_gb300 as pkg
    p = {"fp64": pkg.THC_PREC_FP64, "fp64tc": pkg.THC_PREC_FP64_TC,
         "mixed": pkg.THC_PREC_MIXED}[prec]
    s, Zc, t1, *_ = oracle_case(8, 60, 120, 200, 80, 13)
    out = []
    for poison in ("0", "1"):
        env("THC_POISON_WORKSPACE", poison)
        with context(s, precision=p, **kw) as ctx:
            sig, sig1, E = ctx.residual(Zc, t1)
            Zs, ts, rep = ctx.solve(max_iter=3, raise_on_failure=False)
        out.append((sig, sig1, E, Zs, ts, rep.energy))
    a, b = out
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4]) and a[5] == b[5]
    assert np.isfinite(b[0]).all()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_resumes_bit_identically(prec):
    """10 iterations in one solve = 4 iterations, checkpoint, 6 more (in the
    same context and in a fresh one loaded from the checkpoint)."""
    import paper_2111_11473_gb300 as pkg
    p = {"fp64": pkg.THC_PREC_FP64, "mixed": pkg.THC_PREC_MIXED}[prec]
    s, *_ = oracle_case(7, 37, 70, 90, 45, 11)
    with context(s, precision=p) as ctx:
        Zr, tr, rr = ctx.solve(r_tol=1e-14, max_iter=10, raise_on_failure=False)
    assert rr.status == "THC_ERR_NOT_CONVERGED" and rr.iters == 10
    with context(s, precision=p) as ctx:
        with pytest.raises(pkg.ThcError, match="THC_ERR_ARG"):
            ctx.solve(resume=True, max_iter=1)          # nothing to resume yet
        ctx.solve(r_tol=1e-14, max_iter=4, raise_on_failure=False)
        state = ctx.solve_state()
        Za, ta, ra = ctx.solve(r_tol=1e-14, max_iter=6, resume=True, raise_on_failure=False)
    with context(s, precision=p) as ctx:
        ctx.load_solve_state(state)
        Zb, tb, rb = ctx.solve(r_tol=1e-14, max_iter=6, resume=True, raise_on_failure=False)
    for Z, t, r in ((Za, ta, ra), (Zb, tb, rb)):
        assert r.iters == 10
        assert np.array_equal(Z, Zr) and np.array_equal(t, tr)
        assert r.energy == rr.energy and r.r_norm == rr.r_norm


def test_checkpoint_of_another_system_is_refused():
    import paper_2111_11473_gb300 as pkg
    s, *_ = oracle_case(7, 37, 70, 90, 45, 11)
    s2, *_ = oracle_case(3, 7, 10, 14, 9, 5)
    with context(s) as ctx:
        ctx.solve(r_tol=1e-14, max_iter=2, raise_on_failure=False)
        state = ctx.solve_state()
    with context(s2) as ctx:
        with pytest.raises(pkg.ThcError, match="another system"):
            ctx.load_solve_state(state)
        with pytest.raises(pkg.ThcError, match="THC_ERR_ARG"):
            ctx.load_solve_state(state[:40])
