"""Host logic of the multi-rank benchmark on two gloo ranks (CPU only).

Under torchrun every rank evaluates residuals of its own system (weak
scaling, no collective in the data path); the only collective is the
max-over-ranks reduction of the step time, from which the whole-job rate
is computed.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, _ = bench._dist()
    ms_local = [10.0, 25.0, 17.5, 3.0][r]
    ms_max = bench.max_over_ranks(ms_local, dist, "cpu")
    e2e_max = bench.max_over_ranks(0.5 * ms_local, dist, "cpu")
    rate = bench.whole_job_rate(w, ms_max)
    seed = bench.WORKLOAD["seed"] + r
    dist.barrier()
    q.put((r, w, ms_max, e2e_max, rate, seed))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_max_over_ranks_and_whole_job_rate(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    slowest = max([10.0, 25.0, 17.5, 3.0][:world])
    assert [x[0] for x in res] == list(range(world))
    assert all(x[1] == world for x in res)
    assert all(x[2] == slowest and x[3] == 0.5 * slowest for x in res)
    assert res[0][4] == pytest.approx(world * 1e3 / slowest)
    assert len({x[5] for x in res}) == world       # one distinct system per rank


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_rate(1, 250.0) == pytest.approx(4.0)


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2111_11473_gb300.shard import allreduce_parts, shard_bounds
    # Each rank's "partial residual": the terms of its shard of a sum over
    # 17 items (the role of the Cholesky vectors); its energy part is a
    # number made from the shard's bounds.
    rng = np.random.default_rng(5)
    terms = rng.standard_normal((17, 6, 6))
    terms1 = rng.standard_normal((17, 3, 4))
    lo, hi = shard_bounds(17, rank, world)
    sig = terms[lo:hi].sum(0)
    sig1 = terms1[lo:hi].sum(0)
    e = float(lo * 100 + hi)
    s, s1, et = allreduce_parts(sig, sig1, e)
    q.put((rank, np.abs(s - terms.sum(0)).max(), np.abs(s1 - terms1.sum(0)).max(), et))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_partials_sum_to_the_whole(world):
    """The shards' contiguous blocks cover every item once and the all-reduce
    of the partial (sigma, Omega1, energy) gives the whole sum on every rank."""
    import torch.multiprocessing as mp
    from paper_2111_11473_gb300.shard import shard_bounds
    bounds = [shard_bounds(17, r, world) for r in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == 17
    assert all(bounds[r][1] == bounds[r + 1][0] for r in range(world - 1))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    e_total = sum(lo * 100 + hi for lo, hi in bounds)
    for r, d, d1, e in res:
        assert d < 1e-12 and d1 < 1e-12 and e == e_total
