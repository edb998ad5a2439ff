"""Multi-rank host logic of bench.py (replicas, sharded upset list) on CPU with
two gloo ranks: disjoint slices per step, max-over-ranks time, summed units,
and the gather of the per-variant records to rank 0 (two ranks' campaigns,
gathered, equal one rank's campaign over the whole list)."""
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


def _campaign_records(flips):
    import oracle as O
    from paper_2606_21791_gb300 import synth as S
    sc = S.make_scene(600, 0, S.FP32, 91)
    cams = S.ring_cameras(2, 48, 40)
    m, _, _ = O.campaign(sc.planes, S.FP32, 0, cams, flips)
    return m   # [nvar, 2 views]


def _gather_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    from paper_2606_21791_gb300 import synth as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        flips = S.flips_stratified(14 * 32, 600, 14, S.FP32, 92)[::9]   # 50 upsets
        n = len(flips)
        # uneven shards: batches of 8 dealt round-robin (rank 1 gets fewer rows)
        idx = np.concatenate([np.arange(a, min(a + 8, n)) for a in range(rank * 8, n, 8 * world)])
        rec = _campaign_records(flips[idx])
        got = R.gather_records(idx, rec, n)
        q.put((rank, None if got is None else got.tobytes(), got is None))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_records_in_list_order():
    import numpy as np
    from paper_2606_21791_gb300 import synth as S
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flips = S.flips_stratified(14 * 32, 600, 14, S.FP32, 92)[::9]
    whole = _campaign_records(flips)
    assert out[1][2] and not out[0][2]          # only rank 0 holds the result
    assert out[0][1] == whole.tobytes()          # bit for bit, in list order


def test_gather_without_a_group_reorders_and_checks():
    import numpy as np
    rec = np.zeros((3, 2), dtype=[("a", "<f8"), ("b", "<u4"), ("c", "<u4")])
    rec["b"] = np.arange(6).reshape(3, 2)
    got = R.gather_records([2, 0, 1], rec, 3)
    assert got["b"].tolist() == [[2, 3], [4, 5], [0, 1]]
    with pytest.raises(ValueError):
        R.gather_records([0, 0, 1], rec, 3)
    with pytest.raises(ValueError):
        R.gather_records([0, 1, 5], rec, 3)


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
