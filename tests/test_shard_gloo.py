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
