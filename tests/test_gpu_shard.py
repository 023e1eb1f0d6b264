"""Sharded residual (the multi-GPU split of Sec. III) on one GB300.

A context with shard (s, n) evaluates the shard's part of the residual: the
Cholesky vectors [K s/n, K (s+1)/n) of Algs. 1, 2, 3, 8 and of the Fock
matrix and singles energy, the rows X in [P s/n, P (s+1)/n) of Alg. 6,
Alg. 7 on the last shard and the orbital-energy Fock terms on the first.
The sum of the parts must be the unsharded residual (float64 rounding) and
match the oracle at the float64 bars.  Two processes on the same GPU, each
with its own context, reduce their parts over gloo: the kernels of the two
processes never wait on each other (the reduction runs on the host).
"""
import os
import socket

import numpy as np
import pytest

from tests.gpu_util import context, oracle_case

pytestmark = pytest.mark.gpu

CASE = (7, 37, 70, 90, 45, 11)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


@pytest.fixture(scope="module")
def case():
    return oracle_case(*CASE)


@pytest.mark.parametrize("count", [2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp64tc", "mixed"])
def test_shards_sum_to_the_whole_residual(case, count, prec):
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, sig_ref, r1_ref, E_ref = case
    p = {"fp64": pkg.THC_PREC_FP64, "fp64tc": pkg.THC_PREC_FP64_TC,
         "mixed": pkg.THC_PREC_MIXED}[prec]
    with context(s, precision=p) as c:
        whole = c.residual(Zc, t1)
    parts = []
    for i in range(count):
        with context(s, precision=p, shard=(i, count)) as c:
            parts.append(c.residual(Zc, t1))
    sig = sum(q[0] for q in parts)
    sig1 = sum(q[1] for q in parts)
    E = sum(q[2] for q in parts)
    scale = max(np.abs(whole[0]).max(), np.abs(whole[1]).max())
    d = max(np.abs(sig - whole[0]).max(), np.abs(sig1 - whole[1]).max())
    print(f"{prec} {count} shards: max|sum of parts - whole| / max|sigma| = {d / scale:.2e}")
    assert d < (1e-12 if prec != "mixed" else 1e-5) * scale
    assert abs(E - whole[2]) < (1e-12 if prec != "mixed" else 1e-7)
    if prec != "mixed":
        assert np.abs(sig - sig_ref).max() < 1e-10 and np.abs(sig1 - r1_ref).max() < 1e-10
        assert abs(E - E_ref) < 1e-9


def test_sharded_context_loads_only_its_vectors_and_refuses_solve(case):
    """Vectors outside the shard may be offered slab by slab and are ignored;
    thc_solve needs the whole residual and is refused."""
    import paper_2111_11473_gb300 as pkg
    s, Zc, t1, sig_ref, r1_ref, E_ref = case
    parts = []
    for i in range(2):
        ctx = pkg.Context(s.eps_o, s.eps_v, s.Y, None, s.x, s.z, n_k=s.K, shard=(i, 2))
        for k0 in range(0, s.K, 8):
            ctx.load_cholesky(k0, s.L[k0:k0 + 8])
        ctx.finish_init()
        parts.append(ctx.residual(Zc, t1))
        with pytest.raises(pkg.ThcError) as e:
            ctx.solve(max_iter=2)
        assert "sharded" in str(e.value)
        ctx.close()
    assert np.abs(parts[0][0] + parts[1][0] - sig_ref).max() < 1e-10
    with pytest.raises(pkg.ThcError):
        pkg.Context(s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z, shard=(2, 2))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import __graft_entry__ as g
    g.build()
    from paper_2111_11473_gb300.shard import sharded_residual
    s, Zc, t1, sig_ref, r1_ref, E_ref = oracle_case(*CASE)
    with context(s, shard=(rank, world)) as c:
        sig, sig1, E = sharded_residual(c, Zc, t1)
    q.put((rank, float(np.abs(sig - sig_ref).max()), float(np.abs(sig1 - r1_ref).max()),
           abs(E - E_ref)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_over_gloo_match_the_oracle():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    for r, d, d1, dE in res:
        print(f"rank {r}: max|d sigma| {d:.2e}, max|d Omega1| {d1:.2e}, dE {dE:.2e}")
        assert d < 1e-10 and d1 < 1e-10 and dE < 1e-9
