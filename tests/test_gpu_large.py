"""Paths for systems too large for one array or one block (needs a GB300):
Alg. 6 in blocks of X rows, Cholesky vectors loaded in parts, the packed
virtual-virtual block, and the memory-driven automatic blocking."""
import numpy as np
import pytest

from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu

RES_TOL = 1e-10
E_TOL = 1e-9
MIXED_BOUND = 1e-4   # bf16x3 products, relative to max |sigma|


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.mark.parametrize("x6", [32, 17, 1, 70])
@pytest.mark.parametrize("route", [1, 2])
def test_alg6_x_blocks_match_oracle(x6, route):
    """Blocks of 32 (two full, one ragged of 6), 17, 1 and all 70 rows."""
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(7, 37, 70, 90, 45, 11)
    with context(s, x_block6=x6, alg7_route=route) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    with context(s, alg7_route=route) as ctx:
        sig0, sig10, E0 = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert np.abs(sig1 - r1_ref).max() < RES_TOL
    assert abs(E - E_ref) < E_TOL
    assert np.abs(sig - sig0).max() < 1e-12
    assert np.abs(sig - sig.T).max() < 1e-12 * max(1.0, np.abs(sig).max())


@pytest.mark.parametrize("case,x6,ic", [((8, 60, 120, 200, 80, 13), 32, 0),   # paired kernel, ragged 24
                                        ((8, 60, 120, 200, 80, 13), 64, 0),
                                        ((8, 60, 120, 200, 80, 13), 31, 37),  # odd row blocks
                                        ((7, 37, 70, 90, 45, 11), 32, 0)],    # P % 4 != 0 kernel
                         ids=["P120x32", "P120x64", "P120x31ic37", "P70x32"])
@pytest.mark.parametrize("tcp", [3, 0])
def test_mixed_alg6_x_blocks_within_bound(case, x6, ic, tcp):
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(*case)
    with context(s, precision=pkg.THC_PREC_MIXED, tc_products=tcp, x_block6=x6,
                 alg7_route=1, i_chunk=ic) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    scale = max(np.abs(sig_ref).max(), np.abs(r1_ref).max())
    err = max(np.abs(sig - sig_ref).max(), np.abs(sig1 - r1_ref).max())
    print(f"mixed x6={x6} tc={tcp} {case}: {err / scale:.2e}")
    assert err < (MIXED_BOUND if tcp == 3 else 2e-5) * scale
    assert abs(E - E_ref) < 1e-6 * max(1e-3, abs(E_ref))


def test_memory_budget_forces_blocks_and_grid_chunks():
    """A small workspace budget makes the automatic choice split Alg. 6 into
    X blocks and rebuild G_I per grid chunk; the result does not change."""
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(7, 37, 70, 90, 45, 11)
    with context(s, workspace_bytes=8 << 20) as ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert np.abs(sig1 - r1_ref).max() < RES_TOL
    assert abs(E - E_ref) < E_TOL


def _parts_context(s, parts, **kw):
    import paper_2111_11473_gb300 as pkg
    ctx = pkg.Context(s.eps_o, s.eps_v, s.Y, None, s.x, s.z, n_k=s.K, **kw)
    for k0, k1 in parts:
        ctx.load_cholesky(k0, s.L[k0:k1])
    ctx.finish_init()
    return ctx


@pytest.mark.parametrize("mixed", [False, True])
def test_cholesky_loaded_in_parts_equals_one_array(mixed):
    import paper_2111_11473_gb300 as pkg
    prec = pkg.THC_PREC_MIXED if mixed else pkg.THC_PREC_FP64
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(7, 37, 70, 90, 45, 11)
    with context(s, precision=prec) as ctx:
        want = ctx.residual(Zc, t1)
    # out of order, uneven, one vector loaded twice
    with _parts_context(s, [(20, 45), (0, 7), (7, 20), (3, 4)], precision=prec) as ctx:
        got = ctx.residual(Zc, t1)
        e = ctx.energy(Zc, t1)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])
    assert got[2] == want[2] and e == want[2]


def test_cholesky_loaded_from_device_tensors():
    torch = pytest.importorskip("torch")
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(3, 7, 10, 14, 9, 5)
    import paper_2111_11473_gb300 as pkg
    dev = torch.device("cuda:0")
    ctx = pkg.Context(s.eps_o, s.eps_v, s.Y, None, s.x, s.z, n_k=s.K)
    Ld = torch.from_numpy(s.L).to(dev)
    ctx.load_cholesky(0, Ld[:4])
    ctx.load_cholesky(4, Ld[4:])
    ctx.finish_init()
    with ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    assert np.abs(sig - sig_ref).max() < RES_TOL
    assert abs(E - E_ref) < E_TOL


def test_pending_context_refuses_work():
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, *_ = oracle_case(3, 7, 10, 14, 9, 5)
    ctx = pkg.Context(s.eps_o, s.eps_v, s.Y, None, s.x, s.z, n_k=s.K)
    with ctx:
        with pytest.raises(pkg.ThcError, match="THC_ERR_ARG"):
            ctx.residual(Zc, t1)
        with pytest.raises(pkg.ThcError, match="THC_ERR_ARG"):
            ctx.load_cholesky(5, s.L[:5])              # runs past K = 9
        ctx.load_cholesky(0, s.L[:8])
        with pytest.raises(pkg.ThcError, match="not loaded"):
            ctx.finish_init()                         # vector 8 missing
        ctx.load_cholesky(8, s.L[8:])
        ctx.finish_init()
        with pytest.raises(pkg.ThcError, match="THC_ERR_ARG"):
            ctx.load_cholesky(0, s.L[:1])             # nothing pending any more
        with pytest.raises(pkg.ThcError, match="THC_ERR_ARG"):
            ctx.finish_init()
        ctx.residual(Zc, t1)


def test_device_generated_system_runs():
    """A system generated on the device in slabs goes through the slab loader;
    its residual matches the one of the host-generated system to float32
    accuracy of the Cholesky vectors."""
    torch = pytest.importorskip("torch")
    import paper_2111_11473_gb300 as pkg
    from synth import make_device_system
    case = (7, 37, 70, 90, 45, 11)
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(*case)
    d = make_device_system(*case, device=torch.device("cuda:0"))
    ctx = pkg.Context(d.eps_o, d.eps_v, d.Y, None, d.x, d.z, n_k=d.K)
    for k0, Lk in d.cholesky_slabs(nk=16):
        ctx.load_cholesky(k0, Lk)
    ctx.finish_init()
    with ctx:
        sig, sig1, E = ctx.residual(Zc, t1)
    scale = max(np.abs(sig_ref).max(), np.abs(r1_ref).max())
    assert np.abs(sig - sig_ref).max() < 1e-5 * scale
    assert abs(E - E_ref) < 1e-5 * max(1e-3, abs(E_ref))
