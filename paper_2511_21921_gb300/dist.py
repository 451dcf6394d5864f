"""Host-side logic for running independent boxes on several GPUs.

Boxes are independent problems, so N ranks need no data-path collective: each
rank takes a set of whole boxes (balanced by particle count) and runs them in
one batched call; a single-box workload is replicated (weak scaling).  The only
collective is the max over ranks of the step time.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_boxes(sizes, world: int) -> list[list[int]]:
    """Assign box indices to ``world`` ranks, largest first to the least loaded
    rank (deterministic; ties go to the lower rank)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for b in sorted(range(sizes.size), key=lambda k: (-int(sizes[k]), k)):
        load, r = heapq.heappop(heap)
        out[r].append(b)
        heapq.heappush(heap, (load + int(sizes[b]), r))
    return [sorted(o) for o in out]


def shard_workload(d: dict, rank: int, world: int) -> dict:
    """The part of workload ``d`` that ``rank`` runs: its boxes for a multi-box
    set (with box offsets rebuilt), the whole box otherwise."""
    if "box_off" not in d or world == 1:
        return d
    off = np.asarray(d["box_off"])
    mine = partition_boxes(np.diff(off), world)[rank]
    cols = np.concatenate([np.arange(off[b], off[b + 1]) for b in mine]) if mine else \
        np.zeros(0, dtype=np.int64)
    out = {k: d[k][..., cols] for k in ("x", "v", "u", "h", "m")}
    sz = np.array([off[b + 1] - off[b] for b in mine], dtype=np.int64)
    out["box_off"] = np.concatenate([[0], np.cumsum(sz)]).astype(np.int64)
    out["box_L"] = np.asarray(d["box_L"])[mine] if mine else np.zeros(0)
    out["L"] = d["L"]
    out["boxes"] = np.asarray(mine, dtype=np.int64)
    return out


def max_over_ranks(value: float, device=None) -> float:
    """Max of ``value`` over the default process group (identity when none)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
