"""Replicas across GPUs: the host logic of the data-parallel campaign.

Upsets are independent units (the study runs them data-parallel across devices
with no communication), so N GPUs each hold the scene and its clean state and
take disjoint slices of the upset list.  The cross-rank steps are a barrier
around the timed region, the max/sum of per-rank times and counts, and the
gather of the per-variant records to rank 0 at the end of a campaign, done with
torch.distributed on whatever backend the caller initialised (NCCL on GPUs,
gloo in the CPU tests)."""
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


def gather_records(indices, records, n_total: int, device=None):
    """Collect every rank's per-variant records on rank 0, ordered by upset index.

    indices: int array, the upset index of each local row; records: a numpy
    structured array with one row per index (e.g. the engine's 24-B records,
    one row per variant with the views as a sub-array).  Returns, on rank 0,
    the records of all n_total upsets in list order (every index must come from
    exactly one rank, else ValueError) and None on the other ranks.  Without a
    process group it only reorders the local rows.  The one data collective of
    the replicated campaign: an all-gather of the row counts, then of the
    padded indices and record bytes."""
    import numpy as np
    import torch
    import torch.distributed as dist
    indices = np.asarray(indices, dtype=np.int64).reshape(-1)
    records = np.ascontiguousarray(records)
    if len(indices) != len(records):
        raise ValueError("one record row per index")
    row = records.dtype.itemsize * int(np.prod(records.shape[1:]))
    grouped = dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    if not grouped:
        parts = [(indices, records.view(np.uint8).reshape(len(indices), row))]
    else:
        world = dist.get_world_size()
        n = torch.tensor([len(indices)], dtype=torch.int64, device=device)
        sizes = [torch.zeros_like(n) for _ in range(world)]
        dist.all_gather(sizes, n)
        sizes = [int(s.item()) for s in sizes]
        m = max(max(sizes), 1)
        idx = torch.full((m,), -1, dtype=torch.int64, device=device)
        idx[:len(indices)] = torch.from_numpy(indices).to(device)
        raw = torch.zeros((m, row), dtype=torch.uint8, device=device)
        if len(indices):
            raw[:len(indices)] = torch.from_numpy(records.view(np.uint8).reshape(len(indices), row).copy()).to(device)
        all_idx = [torch.empty_like(idx) for _ in range(world)]
        all_raw = [torch.empty_like(raw) for _ in range(world)]
        dist.all_gather(all_idx, idx)
        dist.all_gather(all_raw, raw)
        if dist.get_rank() != 0:
            return None
        parts = [(all_idx[r][:sizes[r]].cpu().numpy(), all_raw[r][:sizes[r]].cpu().numpy()) for r in range(world)]
    out = np.zeros((n_total, row), dtype=np.uint8)
    seen = np.zeros(n_total, dtype=np.int64)
    for ix, raw in parts:
        if len(ix) and (ix.min() < 0 or ix.max() >= n_total):
            raise ValueError("upset index out of range")
        out[ix] = raw
        np.add.at(seen, ix, 1)
    if not (seen == 1).all():
        raise ValueError("every upset index must come from exactly one rank")
    shape = (n_total,) + records.shape[1:]
    return out.view(records.dtype).reshape(shape)
