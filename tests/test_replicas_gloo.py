"""Multi-rank host logic (replicas / ensemble sharding) with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2001_05234_b300 import inputs as I
from paper_2001_05234_b300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        slowest = R.max_over_ranks(ms)
        sizes = [c.points for c in I.ensemble_cases(count=16, sizes=(16, 24, 32))]
        mine = R.assign_problems(sizes, world)[rank]
        dist.barrier()
        q.put((rank, slowest, mine))
    finally:
        dist.destroy_process_group()


def test_two_ranks_agree_on_slowest_time_and_split_the_ensemble():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    assert all(r[1] == 15.0 for r in results)
    split = [r[2] for r in results]
    allq = sorted(split[0] + split[1])
    assert allq == list(range(16)) and not set(split[0]) & set(split[1])


def test_assign_problems_balances_load():
    sizes = [c.points for c in I.ensemble_cases()]
    parts = R.assign_problems(sizes, 4)
    loads = [sum(sizes[q] for q in p) for p in parts]
    assert sorted(q for p in parts for q in p) == list(range(len(sizes)))
    assert max(loads) - min(loads) <= max(sizes)


def test_aggregate_throughput():
    assert R.aggregate_gpts(10**9, 1000.0, 4) == pytest.approx(4.0)
