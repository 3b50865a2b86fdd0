"""Host side of the z-slab split of one solve (CPU, no GPU): the slab partition and the all-gather
exchange of the elimination pass's numbers, run as two gloo ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2001_05234_b300.zslab import gather_exchange, slab_ranges


@pytest.mark.parametrize("nz,p", [(10, 1), (10, 2), (10, 3), (7, 7), (512, 8), (33, 4)])
def test_slab_ranges_cover_the_column(nz, p):
    r = slab_ranges(nz, p)
    assert r[0][0] == 0 and r[-1][1] == nz
    assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    sizes = [b - a for a, b in r]
    assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    assert sizes == sorted(sizes, reverse=True)


def test_slab_ranges_refuse_too_many_ranks():
    with pytest.raises(ValueError):
        slab_ranges(3, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, nz, ncol, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slabs = slab_ranges(nz, world)
        z0, z1 = slabs[rank]
        # rank-tagged numbers: interface block rank*1000 + index, column piece = the global plane index
        iface = torch.arange(ncol * 10, dtype=torch.float64) + 1000.0 * rank
        col00 = torch.arange(z0, z1, dtype=torch.float64)
        ia, ca = gather_exchange()(iface, col00, slabs)
        want_i = torch.cat([torch.arange(ncol * 10, dtype=torch.float64) + 1000.0 * r for r in range(world)])
        ok = torch.equal(ia, want_i) and torch.equal(ca, torch.arange(nz, dtype=torch.float64))
        q.put((rank, bool(ok)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nz", [9, 12])
def test_gather_exchange_two_gloo_ranks(nz):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, nz, 6, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, True), (1, True)]
