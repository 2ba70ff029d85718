"""GPU parity for the first-order Taylor lookup of the Ewald correction (Sec. 2.2.5, approach 2):
the device-generated Taylor table against the oracle's, the FP64 walk against the oracle walk in
Taylor mode (same MAC, same expansion point), the FP32 walk against the exact series, and the
batched persistent kernel in Taylor mode against the single-grid walk."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I
from tests.gpu_util import e_a, run_gravity

pytestmark = pytest.mark.gpu

BOXES = [((1, 1, 1), (1.0, 1.0, 1.0)), ((1, 1, 1), (1.0, 1.0, 2.0)), ((1, 1, 0), (1.0, 1.0, 4.0)),
         ((1, 1, 0), (1.0, 2.0, 1.0)), ((1, 0, 0), (1.0, 1.0, 1.0))]


def _mesh(bc, box, n=16, seed=0):
    mesh = I.uniform_mesh(n, box=box, bc=bc)
    rng = np.random.default_rng(seed)
    return mesh, np.exp(0.7 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))


@pytest.mark.parametrize("bc,box", BOXES)
def test_taylor_table_matches_oracle(oracle, bc, box):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    mesh, rho = _mesh(bc, box, n=8)
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    n = 17 if bc != (1, 0, 0) else 9
    ts.ewald_field(n)
    tab = ts.ewald_taylor_table()
    ref, _ = oracle.ewald_taylor_table(bc, box, n=n)
    # values: the two FP64 series agree to ~1e-13; the Jacobian divides their differences by 2 eps
    np.testing.assert_allclose(tab[..., :4], ref[..., :4], rtol=1e-11, atol=1e-11 * np.abs(ref[..., :4]).max())
    np.testing.assert_allclose(tab[..., 4:], ref[..., 4:], rtol=0, atol=1e-7 * np.abs(ref[..., 4:]).max())


@pytest.mark.parametrize("bc,box", BOXES[:4])
def test_fp64_taylor_walk_matches_oracle(oracle, bc, box):
    mesh, rho = _mesh(bc, box)
    tab = oracle.ewald_taylor_table(bc, box, n=64)
    p_ref, a_ref, cnt = oracle.gravity_walk(mesh, rho, ewald="taylor", table=tab)
    _, p64, a64, st = run_gravity(mesh, rho, precision="fp64", ewald_n=64, ewald="taylor")
    # the Jacobians differ by ~1e-9 relative (differences of two independent series over 2 eps)
    assert e_a(a64, a_ref).max() < 1e-8
    np.testing.assert_allclose(p64, p_ref, rtol=1e-8, atol=1e-8 * np.abs(p_ref).max())
    assert st["interactions"] == cnt["interactions"]


@pytest.mark.parametrize("bc,box", BOXES)
def test_fp32_taylor_walk_against_exact_series(oracle, bc, box):
    mesh, rho = _mesh(bc, box, n=16, seed=1)
    tg = I.sample_cells(mesh.ncell, 200, seed=2)
    p_ref, a_ref, _ = oracle.gravity_walk(mesh, rho, tg, ewald="series")
    _, p32, a32, _ = run_gravity(mesh, rho, precision="fp32", ewald_n=64 if bc != (1, 0, 0) else 32, ewald="taylor")
    e = e_a(a32[tg], a_ref)
    assert np.median(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2, (np.median(e), e.max())
    dp = (p32[tg] - p32[tg].mean()) - (p_ref - p_ref.mean())
    assert np.median(np.abs(dp)) < 1e-3 * np.abs(p_ref).max()


def test_fp32_taylor_walk_matches_oracle_taylor_walk(oracle):
    bc, box = (1, 1, 0), (1.0, 1.0, 4.0)
    mesh, rho = _mesh(bc, box, seed=3)
    tab = oracle.ewald_taylor_table(bc, box, n=64)
    tg = I.sample_cells(mesh.ncell, 1024, seed=4)
    _, a_ref, _ = oracle.gravity_walk(mesh, rho, tg, ewald="taylor", table=tab)
    _, _, a32, _ = run_gravity(mesh, rho, precision="fp32", ewald_n=64, ewald="taylor")
    e = e_a(a32[tg], a_ref)
    assert np.median(e) <= 1e-5 and np.quantile(e, 0.99) <= 1e-4, (np.median(e), e.max())


def test_batched_taylor_matches_single_grid():
    import torch
    from paper_1708_06142_gb300.treesolver import Batch, TreeSolver
    grids = [_mesh((1, 1, 1), (1.0, 1.0, 1.0), n=16, seed=5), _mesh((1, 1, 0), (1.0, 1.0, 4.0), n=16, seed=6),
             _mesh((0, 0, 0), (1.0, 1.0, 1.0), n=16, seed=7)]
    solvers, pots, accs, refs = [], [], [], []
    for mesh, rho in grids:
        ts = TreeSolver(0)
        ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
        if any(mesh.bc):
            ts.ewald_field(64)
        p1 = torch.empty(mesh.ncell, device="cuda")
        a1 = torch.empty(mesh.ncell, 3, device="cuda")
        ts.gravity_walk(p1, a1, ewald="taylor")
        ts.sync()
        refs.append(a1.cpu().numpy().astype(np.float64))
        solvers.append(ts)
        pots.append(torch.empty(mesh.ncell, device="cuda"))
        accs.append(torch.empty(mesh.ncell, 3, device="cuda"))
    b = Batch(solvers)
    b.run(gravity=solvers[0].gravity_params(ewald="taylor"), pots=pots, accs=accs)
    b.sync()
    for a, ref in zip(accs, refs):
        assert e_a(a.cpu().numpy().astype(np.float64), ref).max() < 1e-5
