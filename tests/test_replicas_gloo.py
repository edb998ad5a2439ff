"""Multi-rank host logic of bench.py (replicas, sharded upset list) on CPU with
two gloo ranks: disjoint slices per step, max-over-ranks time, summed units."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2606_21791_gb300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slices = [R.step_slice(step, rank, world, 64, 20_000) for step in range(40)]
        t, u = R.aggregate(1.0 + rank, 64 * 40)
        dist.barrier()
        q.put((rank, slices, t, u))
    finally:
        dist.destroy_process_group()


def test_step_slices_partition_the_list():
    world, batch, n = 4, 64, 20_000
    seen = set()
    for step in range(n // (batch * world)):
        for rank in range(world):
            a, b = R.step_slice(step, rank, world, batch, n)
            assert 0 <= a < b <= n
            rng = set(range(a, b))
            assert not (rng & seen)
            seen |= rng
    with pytest.raises(ValueError):
        R.step_slice(0, 0, 1, 100, 50)


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    s0 = out[0][1]
    s1 = out[1][1]
    for a, b in zip(s0, s1):
        assert a[1] <= b[0] or b[1] <= a[0]          # disjoint within a step
    assert all(r[2] == 2.0 for r in out)             # max over ranks
    assert all(r[3] == 2 * 64 * 40 for r in out)     # units summed
