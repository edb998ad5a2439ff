"""Host side of the support guard's health signal (Algorithm 1, last step).

Each clamp of the guard is the detection of an out-of-range stored value, so
the guard reports how many it made instead of silently absorbing them: per
frame, the clamp counts of the nodes (each guarding the primitives it holds)
are summed, and when the sum exceeds a health threshold the host raises a
parity / scrub alert -- a degrading device must not be masked by the clamp.

The per-node counts come from `gs_guard` / `gs_guard_bitmap` (the count added to
`dev_clamps`) or from the serving loop's guarded storm frames.  The sum over
nodes uses torch.distributed when a process group is up (any backend: NCCL on
GPUs, gloo in the CPU tests); without one it is the local count.  This sum is
the only exchange step of the guard.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Optional


@dataclass(frozen=True)
class Alert:
    frame: int        # index of the frame (0-based, counted by this monitor)
    total: int        # clamps summed over the nodes in that frame
    threshold: int    # the health threshold it exceeded


def sum_over_nodes(local: int, device=None) -> int:
    """Sum of every node's `local` count (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(local)
    t = torch.tensor([int(local)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


class GuardHealth:
    """Per-frame health check of the guard: `frame(local_clamps)` sums the
    nodes' clamp counts and records (and reports to `on_alert`) an alert when
    the sum is strictly above `threshold`.  Every node calls `frame` once per
    frame, so every node sees the same totals and the same alerts."""

    def __init__(self, threshold: int, on_alert: Optional[Callable[[Alert], None]] = None):
        if int(threshold) < 0:
            raise ValueError("the health threshold is a clamp count (>= 0)")
        self.threshold = int(threshold)
        self.on_alert = on_alert
        self.frames = 0
        self.total_clamps = 0
        self.alerts: List[Alert] = []

    def frame(self, local_clamps: int, device=None) -> int:
        if int(local_clamps) < 0:
            raise ValueError("a clamp count is >= 0")
        total = sum_over_nodes(local_clamps, device)
        index = self.frames
        self.frames += 1
        self.total_clamps += total
        if total > self.threshold:
            alert = Alert(index, total, self.threshold)
            self.alerts.append(alert)
            if self.on_alert is not None:
                self.on_alert(alert)
        return total
