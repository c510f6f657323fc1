"""The multi-GPU form on CPU: 2 gloo ranks check that the bench's sharding gives
every unit to exactly one rank and that the timed region is the max over ranks.
No data-path collective exists: only the timing barrier and max."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, total_units, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard_units(total_units, rank, world)
        bench.barrier(world)
        t = bench.max_over_ranks(float(10 + rank * 5), world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out_q.put((rank, mine, t, gathered))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,total", [(2, 2), (2, 7), (2, 256)])
def test_two_rank_sharding_and_max(world, total):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, total, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    units = sorted(u for _, mine, _, _ in res for u in mine)
    assert units == list(range(total))
    for _, _, t, _ in res:
        assert t == 10 + (world - 1) * 5


def test_single_rank_helpers():
    assert bench.shard_units(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
