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
