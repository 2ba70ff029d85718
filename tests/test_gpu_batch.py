"""Batched persistent execution: many independent grids in one persistent kernel (optionally a
captured CUDA graph) must give the same results as walking each grid with its own kernels."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _grids():
    out = []
    rng = np.random.default_rng(0)
    for k, (n, bc, box) in enumerate([(16, (0, 0, 0), (1, 1, 1)), (32, (1, 1, 1), (1, 1, 1)),
                                      (16, (1, 1, 0), (1, 1, 2)), (32, (0, 0, 0), (1, 1, 1)),
                                      (8, (1, 1, 1), (1, 1, 1))]):
        mesh = I.uniform_mesh(n, box=box, bc=bc)
        rho = np.exp(0.5 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))
        out.append((mesh, rho))
    out.append(I.plummer_amr(seed=3, max_level=4))
    return out


def _setup(grids):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    solvers, dens = [], []
    for mesh, rho in grids:
        ts = TreeSolver(0)
        d = torch.from_numpy(rho.reshape(-1)).cuda()
        ts.tree_build(mesh, d)
        if any(mesh.bc):
            ts.ewald_field(32)
        solvers.append(ts)
        dens.append(d)
    return solvers, dens


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_gravity_and_columns_match_single_grid_walks(mode):
    import torch
    from paper_1708_06142_gb300.treesolver import Batch
    grids = _grids()
    solvers, dens = _setup(grids)
    gp = solvers[0].gravity_params(theta=0.5, zero_mean=True)
    cp = solvers[0].column_params(n_side=2, theta=0.5)
    ref_p, ref_a, ref_c = [], [], []
    for ts, (mesh, _) in zip(solvers, grids):
        p = torch.empty(mesh.ncell, device="cuda")
        a = torch.empty(mesh.ncell, 3, device="cuda")
        c = torch.empty(mesh.ncell, 48, device="cuda")
        ts.gravity_walk(p, a, gp)
        ts.column_walk(c, cp)
        ts.sync()
        ref_p.append(p.cpu().numpy()); ref_a.append(a.cpu().numpy()); ref_c.append(c.cpu().numpy())
    b = Batch(solvers)
    b.set_mode(mode, 3)
    pots = [torch.full((m.ncell,), np.nan, device="cuda") for m, _ in grids]
    accs = [torch.full((m.ncell, 3), np.nan, device="cuda") for m, _ in grids]
    cols = [torch.full((m.ncell, 48), np.nan, device="cuda") for m, _ in grids]
    for use_graph in (False, True, True):   # direct, capture, replay
        b.run(gp, pots, accs, cp, cols, densities=dens, use_graph=use_graph)
        st = b.sync()
        assert st["cells"] == sum(m.ncell for m, _ in grids)
        assert st["items"] == 2 * st["cells"] // 32
        for k in range(len(grids)):
            # potentials after the zero-mean shift sit near 0: compare on the scale of the potential (O(1))
            np.testing.assert_allclose(pots[k].cpu().numpy(), ref_p[k], rtol=1e-6, atol=1e-6 * max(np.abs(ref_p[k]).max(), 1.0))
            np.testing.assert_allclose(accs[k].cpu().numpy(), ref_a[k], rtol=1e-6, atol=1e-6 * np.abs(ref_a[k]).max())
            np.testing.assert_allclose(cols[k].cpu().numpy(), ref_c[k], rtol=1e-6, atol=1e-6 * np.abs(ref_c[k]).max())


def test_graph_replay_reads_new_densities_and_tuning():
    import torch
    from paper_1708_06142_gb300.treesolver import Batch
    grids = _grids()[:3]
    solvers, dens = _setup(grids)
    gp = solvers[0].gravity_params(theta=0.5)
    b = Batch(solvers)
    pots = [torch.empty(m.ncell, device="cuda") for m, _ in grids]
    accs = [torch.empty(m.ncell, 3, device="cuda") for m, _ in grids]
    b.run(gp, pots, accs, densities=dens, use_graph=True)
    b.sync()
    first = [p.cpu().numpy().copy() for p in pots]
    for d in dens:
        d.mul_(2.0)                       # same buffers, new contents: the replay rebuilds the trees
    b.run(gp, pots, accs, densities=dens, use_graph=True)
    b.sync()
    for p, f in zip(pots, first):
        np.testing.assert_allclose(p.cpu().numpy(), 2 * f, rtol=1e-5, atol=1e-6 * np.abs(f).max())
    for chunk, ctas in ((1, 1), (16, 0), (64, 2)):
        b.set_tuning(chunk, ctas)
        b.run(gp, pots, accs, densities=dens, use_graph=True)
        b.sync()
        for p, f in zip(pots, first):
            np.testing.assert_allclose(p.cpu().numpy(), 2 * f, rtol=1e-5, atol=1e-6 * np.abs(f).max())


def test_autotune_walk_picks_a_grouping():
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver, autotune_walk
    mesh, rho = I.plummer_amr(seed=2, max_level=5)
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    pot = torch.empty(mesh.ncell, device="cuda")
    acc = torch.empty(mesh.ncell, 3, device="cuda")
    best, ms = autotune_walk(ts, pot, acc, ts.gravity_params(theta=0.5))
    assert best in (1, 2, 4) and ms[[1, 2, 4].index(best)] == ms.min() and (ms > 0).all()


def test_per_grid_mode_recaptures_on_new_parameters():
    # mode 1 bakes the descriptors into the captured graph: a new theta must reach the replay
    import torch
    from paper_1708_06142_gb300.treesolver import Batch
    grids = _grids()[:4]
    solvers, dens = _setup(grids)
    b = Batch(solvers)
    b.set_mode(1, 2)
    pots = [torch.empty(m.ncell, device="cuda") for m, _ in grids]
    accs = [torch.empty(m.ncell, 3, device="cuda") for m, _ in grids]
    for theta in (0.5, 0.35, 0.35):
        gp = solvers[0].gravity_params(theta=theta)
        b.run(gp, pots, accs, densities=dens, use_graph=True)
        b.sync()
        for ts, (mesh, _), a in zip(solvers, grids, accs):
            ref = torch.empty(mesh.ncell, 3, device="cuda")
            ts.gravity_walk(torch.empty(mesh.ncell, device="cuda"), ref, gp)
            ts.sync()
            np.testing.assert_allclose(a.cpu().numpy(), ref.cpu().numpy(), rtol=1e-6,
                                       atol=1e-6 * np.abs(ref.cpu().numpy()).max())

