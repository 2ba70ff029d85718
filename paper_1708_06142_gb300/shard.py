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


# ---------------------------------------------------------------- one mesh over several ranks
#
# A rank owns a contiguous range of leaf-blocks in block order (the Morton order of the meshes of
# Sec. 2).  Per step: the densities of all ranges are gathered (every rank then builds the whole
# tree: a replicated build, the exchange of the paper's Sec. 2.1 communication step), each rank
# walks its own range, and, for a periodic potential, the FP64 sums (sum dV phi, sum dV) of all
# ranges are all-reduced so that every rank subtracts the same mean.  The interactions of each
# block in this walk are all-reduced too and give the next step's ranges (Sec. 2.2.6: balance on
# per-block work).

def block_ranges(costs: Sequence[float], world: int) -> list[tuple[int, int]]:
    """Split blocks 0..n-1 into `world` contiguous ranges [begin, end) of near-equal total cost.

    Range r ends at the block boundary nearest to the cost quantile r/world (ties: the earlier
    boundary); boundaries never decrease, so ranges may be empty when one block outweighs a whole
    share.  Costs <= 0 everywhere fall back to equal block counts.  Deterministic: every rank
    computes the same ranges from the same costs."""
    if world < 1:
        raise ValueError(f"bad world {world}")
    n = len(costs)
    c = [max(0.0, float(x)) for x in costs]
    total = sum(c)
    if total <= 0.0:
        c = [1.0] * n
        total = float(n)
    prefix = [0.0]
    for x in c:
        prefix.append(prefix[-1] + x)
    bounds = [0]
    j = 0
    for r in range(1, world):
        target = total * r / world
        while j < n and prefix[j + 1] < target:
            j += 1
        # boundary j (before block j) or j + 1 (after it): the nearer to the target
        b = j if (j >= n or target - prefix[j] <= prefix[j + 1] - target) else j + 1
        bounds.append(max(b, bounds[-1]))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def gather_ranges(local, ranges, group=None):
    """All-gather of per-range slices: `local` is this rank's slice (a 1-D torch tensor of
    ranges[rank] = [begin, end) elements), the result the concatenation of all ranks' slices in rank
    order.  Slices are padded to the longest for the collective (equal sizes are required)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    sizes = [e - b for b, e in ranges]
    if local.numel() != sizes[dist.get_rank(group)]:
        raise ValueError("local slice does not match this rank's range")
    pad = torch.zeros(max(sizes), dtype=local.dtype, device=local.device)
    pad[:local.numel()] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][:sizes[r]] for r in range(world)])


def all_reduce_sum(values, device=None, group=None):
    """FP64 sum over ranks of a small host vector (the zero-mean sums, per-block counts)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(values, dtype=np.float64), device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def partitioned_gravity_step(ts, mesh, rho_local, ranges, rank, params, pot, acc, zero_mean=False, first=True,
                             ewald_n=64, device=None, group=None):
    """One step of one mesh partitioned over the ranks of the default group: gather the densities
    (this rank holds rho_local, the FP64 densities of its range's cells), build the whole tree,
    walk this rank's range into the full-size pot / acc, subtract the global volume-weighted mean of
    the potential when zero_mean is set.  `first`: ingest the mesh (and tabulate the Ewald field
    for periodic axes).  Returns the interactions of every block in this walk (summed over ranks),
    the cost of the next step's ranges."""
    import numpy as np
    b, e = ranges[rank]
    rho = gather_ranges(rho_local, [(x * 512, y * 512) for x, y in ranges], group=group)
    ts.tree_build(mesh if first else None, rho.to(pot.device))
    if first and any(mesh.bc):
        ts.ewald_field(ewald_n)
    ts.gravity_walk_range(pot, acc, b, e, params)
    if zero_mean:
        s = all_reduce_sum(ts.potential_sums(pot, b, e), device=device, group=group)
        ts.potential_shift(pot, b, e, s[0] / s[1])
    counts = np.zeros(mesh.nleaf)
    counts[b:e] = ts.walk_block_counts()[b:e]
    return all_reduce_sum(counts, device=device, group=group)
