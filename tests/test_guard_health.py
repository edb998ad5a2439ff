"""The guard's health signal (Algorithm 1, last step) on the host: clamp counts
summed over the nodes each frame, an alert strictly above the threshold, the
same totals and alerts on every node (two gloo ranks on CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2606_21791_gb300 import health as HL


def test_single_node_alerts_strictly_above_the_threshold():
    seen = []
    h = HL.GuardHealth(5, on_alert=seen.append)
    totals = [h.frame(c) for c in (0, 5, 6, 1, 40)]
    assert totals == [0, 5, 6, 1, 40]
    assert h.frames == 5 and h.total_clamps == 52
    assert [a.frame for a in h.alerts] == [2, 4] and seen == h.alerts
    assert all(a.threshold == 5 for a in h.alerts) and [a.total for a in h.alerts] == [6, 40]


def test_zero_threshold_alerts_on_any_clamp_and_bad_inputs_are_refused():
    h = HL.GuardHealth(0)
    h.frame(0)
    assert not h.alerts
    h.frame(1)
    assert len(h.alerts) == 1
    with pytest.raises(ValueError):
        HL.GuardHealth(-1)
    with pytest.raises(ValueError):
        h.frame(-3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


# per-frame clamp counts of each node: node 0 and node 1
_COUNTS = [(0, 0), (3, 4), (10, 0), (2, 2), (0, 9)]
_THRESHOLD = 6


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        h = HL.GuardHealth(_THRESHOLD)
        totals = [h.frame(c[rank]) for c in _COUNTS]
        q.put((rank, totals, [(a.frame, a.total) for a in h.alerts], h.total_clamps))
    finally:
        dist.destroy_process_group()


def test_two_gloo_nodes_sum_and_agree():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_totals = [a + b for a, b in _COUNTS]
    want_alerts = [(i, t) for i, t in enumerate(want_totals) if t > _THRESHOLD]
    assert want_alerts == [(1, 7), (2, 10), (4, 9)]
    for rank, totals, alerts, total in out:
        assert totals == want_totals
        assert alerts == want_alerts
        assert total == sum(want_totals)
