"""Replicas across GPUs: the host logic of the data-parallel campaign.

Upsets are independent units (the study runs them data-parallel across devices
with no communication), so N GPUs each hold the scene and its clean state and
take disjoint slices of the upset list.  The only cross-rank steps are a
barrier around the timed region and the max/sum of per-rank times and counts,
done with torch.distributed on whatever backend the caller initialised (NCCL on
GPUs, gloo in the CPU tests)."""
from __future__ import annotations


def step_slice(step: int, rank: int, world: int, batch: int, nflips: int) -> tuple[int, int]:
    """[start, stop) of the upsets that `rank` evaluates at `step`: the global
    batch index step * world + rank walks the list in order, wrapping around."""
    if batch > nflips:
        raise ValueError("batch larger than the upset list")
    span = nflips - nflips % batch if nflips % batch else nflips
    start = ((step * world + rank) * batch) % span
    return start, start + batch


def aggregate(local_seconds: float, local_units: int, device=None):
    """(max seconds over ranks, sum of units over ranks); identity without a
    process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_seconds), int(local_units)
    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())
