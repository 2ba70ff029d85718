"""One mesh partitioned over ranks, run as 2 and 3 virtual ranks one after another on one GPU (each
rank a context of its own with a replicated tree build, walking its range of leaf-blocks): the
assembled result equals the unpartitioned walk bit for bit, the per-block interaction counts of
the ranges add up to the whole walk's, and the zero mean over ranks matches the single-context
zero mean."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _meshes():
    mesh, rho = I.plummer_amr(seed=1, max_level=5)
    box = I.uniform_mesh(32, bc=(1, 1, 1))
    rho_box = np.exp(0.8 * np.random.default_rng(2).standard_normal((box.nleaf, 8, 8, 8)))
    return [("amr", mesh, rho), ("periodic3p", box, rho_box)]


MESHES = _meshes()


@pytest.mark.parametrize("name,mesh,rho", MESHES, ids=[m[0] for m in MESHES])
@pytest.mark.parametrize("world", [2, 3])
def test_virtual_ranks_equal_unpartitioned_walk(name, mesh, rho, world):
    import torch
    from paper_1708_06142_gb300.shard import block_ranges
    from paper_1708_06142_gb300.treesolver import TreeSolver
    d = torch.from_numpy(np.ascontiguousarray(rho).reshape(-1)).cuda()
    periodic = any(mesh.bc)
    kw = dict(mac="bh", theta=0.5)
    # the unpartitioned reference
    ref = TreeSolver(0)
    ref.tree_build(mesh, d)
    if periodic:
        ref.ewald_field(32)
    p_ref = torch.empty(mesh.ncell, device="cuda")
    a_ref = torch.empty(mesh.ncell, 3, device="cuda")
    ref.gravity_walk(p_ref, a_ref, zero_mean=periodic, **kw)
    ref.sync()
    n_int = ref.stats()["interactions"]
    # first step: ranges of equal cell counts; second step: ranges from the first step's counts
    costs = np.ones(mesh.nleaf)
    for step in range(2):
        ranges = block_ranges(costs, world)
        pot = torch.zeros(mesh.ncell, device="cuda")
        acc = torch.zeros(mesh.ncell, 3, device="cuda")
        counts = np.zeros(mesh.nleaf, dtype=np.int64)
        sums = np.zeros(2)
        ranks = []
        for r, (b, e) in enumerate(ranges):
            ts = TreeSolver(0)
            ts.tree_build(mesh, d)                  # replicated build from the gathered densities
            if periodic:
                ts.ewald_field(32)
            p = torch.zeros(mesh.ncell, device="cuda")
            a = torch.zeros(mesh.ncell, 3, device="cuda")
            ts.gravity_walk_range(p, a, b, e, **kw)
            ts.sync()
            counts[b:e] = ts.walk_block_counts()[b:e]
            sums += ts.potential_sums(p, b, e)      # stands in for the all-reduce over ranks
            ranks.append((ts, p, a))
        for r, (b, e) in enumerate(ranges):
            ts, p, a = ranks[r]
            if periodic:
                ts.potential_shift(p, b, e, sums[0] / sums[1])
                ts.sync()
            pot[b * 512:e * 512] = p[b * 512:e * 512]
            acc[b * 512:e * 512] = a[b * 512:e * 512]
        assert int(counts.sum()) == n_int
        assert torch.equal(acc, a_ref), (name, world, step)
        if periodic:
            # the mean is summed in another order than the single-context kernel's: ~1 ulp of phi
            np.testing.assert_allclose(pot.cpu().numpy(), p_ref.cpu().numpy(), rtol=0,
                                       atol=2e-7 * float(p_ref.abs().max()))
        else:
            assert torch.equal(pot, p_ref), (name, world, step)
        costs = counts.astype(float)
    # ranges cut on the measured per-block work are at least as balanced as equal block counts
    load = lambda rs: max(costs[b:e].sum() for b, e in rs)
    assert load(block_ranges(costs, world)) <= load(block_ranges(np.ones(mesh.nleaf), world))


def test_range_walk_arguments():
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver, TSError
    mesh, rho = I.sphere_32(ncell_axis=16)
    ts = TreeSolver(0)
    ts.ncell = mesh.ncell
    pot = torch.zeros(mesh.ncell, device="cuda")
    acc = torch.zeros(mesh.ncell, 3, device="cuda")
    with pytest.raises(TSError) as e:
        ts.gravity_walk_range(pot, acc, 0, 1)
    assert e.value.status == 5
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    with pytest.raises(TSError) as e:
        ts.walk_block_counts()
    assert e.value.status == 5
    for b, e_ in ((-1, 2), (3, 2), (0, mesh.nleaf + 1)):
        with pytest.raises(TSError) as e:
            ts.gravity_walk_range(pot, acc, b, e_)
        assert e.value.status == 1
    with pytest.raises(TSError) as e:
        ts.gravity_walk_range(pot, acc, 0, 2, zero_mean=True)
    assert e.value.status == 1
    ts.gravity_walk_range(pot, acc, 2, 2)              # empty range: nothing written
    ts.sync()
    assert float(pot.abs().max()) == 0.0
    assert (ts.walk_block_counts() == 0).all()
    with pytest.raises(TSError) as e:
        ts.potential_shift(pot, 0, 1, float("nan"))
    assert e.value.status == 1
