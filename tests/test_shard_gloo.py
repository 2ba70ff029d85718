"""Multi-rank sharding of independent grids, on CPU ranks over the gloo backend (world size 2)."""
import os
import socket

import numpy as np
import pytest

from paper_1708_06142_gb300.shard import grids_of_rank, max_over_ranks, weak_throughput

COSTS = [32 ** 3 * 8 ** (g % 3) for g in range(13)]   # cell counts of grids of side 32, 64, 128


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_once_and_balances(world):
    parts = [grids_of_rank(COSTS, r, world) for r in range(world)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(COSTS)))
    loads = [sum(COSTS[i] for i in p) for p in parts]
    # LPT: no rank exceeds the mean load by more than the largest single grid
    assert max(loads) <= sum(COSTS) / world + max(COSTS)
    assert all(p == sorted(p) for p in parts)


def test_partition_edge_cases():
    assert grids_of_rank([], 0, 2) == []
    assert grids_of_rank([5.0], 1, 2) == []
    assert grids_of_rank([5.0], 0, 2) == [0]
    with pytest.raises(ValueError):
        grids_of_rank(COSTS, 2, 2)
    with pytest.raises(ValueError):
        grids_of_rank(COSTS, 0, 0)
    with pytest.raises(ValueError):
        weak_throughput([1.0], 0.0)
    assert max_over_ranks(3.5) == 3.5   # no process group: identity


def _grid_mass(g):
    from paper_1708_06142_gb300 import inputs
    n = 8 * 2 ** (g % 2)
    mesh = inputs.uniform_mesh(n)
    rho = np.random.default_rng(g).lognormal(size=(mesh.ncell,))
    return float(rho.sum()) / mesh.ncell


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [8 ** 3 * 8 ** (g % 2) for g in range(7)]
        mine = grids_of_rank(costs, rank, world)
        res = {g: _grid_mass(g) for g in mine}
        gathered = [None] * world
        dist.all_gather_object(gathered, res)
        t_max = max_over_ranks(1.0 + rank)
        units = [sum(costs[g] for g in grids_of_rank(costs, r, world)) for r in range(world)]
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([t_max, weak_throughput(units, t_max), len(mine)] +
                         [gathered[r].get(g, np.nan) if g in gathered[r] else np.nan
                          for r in range(world) for g in range(7)]))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_gloo_two_ranks_shard_and_reduce(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    serial = [_grid_mass(g) for g in range(7)]
    costs = [8 ** 3 * 8 ** (g % 2) for g in range(7)]
    for rank in range(world):
        v = np.load(tmp_path / f"r{rank}.npy")
        assert v[0] == 2.0                                  # max over ranks of 1 + rank
        assert v[1] == pytest.approx(sum(costs) / 2.0)      # all units / slowest time
        got = v[3:].reshape(world, 7)
        # every grid computed by exactly one rank, with the serial result
        have = ~np.isnan(got)
        assert (have.sum(0) == 1).all()
        np.testing.assert_array_equal(got[have.argmax(0), np.arange(7)], serial)
        assert int(v[2]) == have[rank].sum()


# ---------------------------------------------------------------- one mesh over several ranks

@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_block_ranges_cover_contiguously_and_balance(world):
    from paper_1708_06142_gb300.shard import block_ranges
    rng = np.random.default_rng(world)
    costs = rng.lognormal(0.0, 1.0, 300)
    rs = block_ranges(costs, world)
    assert rs[0][0] == 0 and rs[-1][1] == 300
    assert all(rs[r][1] == rs[r + 1][0] for r in range(world - 1))
    loads = [costs[b:e].sum() for b, e in rs]
    # each boundary is the nearest block boundary to its cost quantile
    assert max(loads) <= costs.sum() / world + 2 * costs.max()
    # deterministic
    assert rs == block_ranges(list(costs), world)


def test_block_ranges_edge_cases():
    from paper_1708_06142_gb300.shard import block_ranges
    assert block_ranges([], 2) == [(0, 0), (0, 0)]
    assert block_ranges([0.0, 0.0, 0.0, 0.0], 2) == [(0, 2), (2, 4)]      # no cost: equal counts
    assert block_ranges([1.0] * 10, 3) == [(0, 3), (3, 7), (7, 10)]
    assert block_ranges([10.0, 1, 1, 1, 1], 2) == [(0, 1), (1, 5)]
    with pytest.raises(ValueError):
        block_ranges([1.0], 0)


def _partition_rank(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    from paper_1708_06142_gb300.shard import all_reduce_sum, block_ranges, gather_ranges
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nleaf = 37
        rng = np.random.default_rng(0)                      # the same data on every rank
        rho = rng.lognormal(size=nleaf * 512)
        pot = rng.standard_normal(nleaf * 512)
        vol = np.repeat(rng.uniform(0.5, 2.0, nleaf), 512)
        costs = rng.integers(1, 1000, nleaf).astype(float)
        ranges = block_ranges(costs, world)
        b, e = ranges[rank]
        # the exchange before the walk: every rank ends up with all blocks' densities
        full = gather_ranges(torch.from_numpy(rho[b * 512:e * 512]), [(x * 512, y * 512) for x, y in ranges])
        # the zero-mean sums of this rank's range, summed over ranks in FP64
        s = all_reduce_sum([(vol * pot)[b * 512:e * 512].sum(), vol[b * 512:e * 512].sum()])
        # per-block counts of the own range, summed over ranks into the next step's costs
        cnt = np.zeros(nleaf)
        cnt[b:e] = costs[b:e] + rank
        c = all_reduce_sum(cnt)
        np.save(os.path.join(out_dir, f"p{rank}.npy"), np.concatenate([full.numpy(), s, c]))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_mesh_partition_exchanges(tmp_path):
    import torch.multiprocessing as mp
    from paper_1708_06142_gb300.shard import block_ranges
    world = 2
    mp.start_processes(_partition_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    nleaf = 37
    rng = np.random.default_rng(0)
    rho = rng.lognormal(size=nleaf * 512)
    pot = rng.standard_normal(nleaf * 512)
    vol = np.repeat(rng.uniform(0.5, 2.0, nleaf), 512)
    costs = rng.integers(1, 1000, nleaf).astype(float)
    ranges = block_ranges(costs, world)
    want_c = costs.copy()
    for r, (b, e) in enumerate(ranges):
        want_c[b:e] += r
    for rank in range(world):
        v = np.load(tmp_path / f"p{rank}.npy")
        np.testing.assert_array_equal(v[:rho.size], rho)           # gathered densities, in block order
        s = v[rho.size:rho.size + 2]
        assert s[0] / s[1] == pytest.approx((vol * pot).sum() / vol.sum(), rel=1e-12, abs=1e-15)
        np.testing.assert_array_equal(v[rho.size + 2:], want_c)
