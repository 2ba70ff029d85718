"""Data-parallel sharding of independent grids over ranks (one process per GPU).

The gravity and column walks of one grid read only that grid's tree (Sec. 2.1 builds one tree per
grid and walks it per target cell), so grids never exchange data: N ranks take disjoint subsets
of the grids, each runs its subset with no collective on the data path, and the only collective is
the max over ranks of a timed region's length (weak scaling).

Host logic only; it runs the same under the gloo (CPU) and nccl (GPU) process-group backends.
"""
from __future__ import annotations

import heapq
from typing import Sequence


def grids_of_rank(costs: Sequence[float], rank: int, world: int) -> list[int]:
    """Indices of the grids that `rank` of `world` processes.

    Longest-processing-time-first assignment on `costs` (e.g. the cell count of each grid, the
    walk being linear in the number of target cells): grids are taken in order of decreasing
    cost, ties by index, and each goes to the rank with the smallest load so far, ties by rank.
    Deterministic, so every rank computes the same partition without communicating.  The
    returned indices are sorted ascending.  Raises ValueError on a bad rank/world.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of world {world}")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """Max of `value` over all ranks of the default process group (the value itself when no group
    is initialised).  `device` is where the reduction tensor lives: a CUDA device under nccl,
    None (CPU) under gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_throughput(units_per_rank: Sequence[float], max_seconds: float) -> float:
    """Whole-job throughput: the units every rank processed divided by the slowest rank's time."""
    if max_seconds <= 0:
        raise ValueError("non-positive time")
    return float(sum(units_per_rank)) / max_seconds
