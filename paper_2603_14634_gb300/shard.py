"""Scene sharding across ranks (one GPU per process).

Scenes are independent, so a batch is split across ranks with no exchange on
the data path: greedy longest-processing-time assignment by particle count
(every scene, largest first, goes to the least loaded rank).  The only
cross-rank traffic is host-side: a barrier around the timed region, the
max of the ranks' times and the gather of per-rank results or metrics.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence


def lpt_partition(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Indices of `sizes` per rank; loads differ by at most max(sizes)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]), r))
    return [sorted(p) for p in parts]


def gather_to_rank0(obj, dist=None):
    """All ranks' objects on rank 0 (list in rank order), None elsewhere."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out if dist.get_rank() == 0 else None


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (e.g. the timed region's length)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
