"""GPU parity for periodic and mixed BCs: the device-generated FP64 Ewald correction table against
the oracle's table, and the walks against the oracle walk with the same table (table mode) and with
the exact series per interaction."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I
from tests.gpu_util import e_a, run_gravity

pytestmark = pytest.mark.gpu

BOXES = [((1, 1, 1), (1.0, 1.0, 1.0)), ((1, 1, 1), (1.0, 1.0, 2.0)), ((1, 1, 0), (1.0, 1.0, 4.0)),
         ((1, 0, 0), (1.0, 1.0, 1.0))]


def _mesh(bc, box, n=16, seed=0):
    mesh = I.uniform_mesh(n, box=box, bc=bc)
    rng = np.random.default_rng(seed)
    return mesh, np.exp(0.7 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))


@pytest.mark.parametrize("bc,box", BOXES)
def test_table_matches_oracle_table(oracle, bc, box):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    mesh, rho = _mesh(bc, box, n=8)
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    n = 24 if bc != (1, 0, 0) else 12
    ts.ewald_field(n)
    tab, ext = ts.ewald_table()
    ref, rext = oracle.ewald_table(bc, box, n=n)
    np.testing.assert_allclose(ext, rext, rtol=1e-15)
    np.testing.assert_allclose(tab, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("bc,box", BOXES[:3])
def test_fp64_walk_matches_oracle_table_walk(oracle, bc, box):
    mesh, rho = _mesh(bc, box)
    tab = oracle.ewald_table(bc, box, n=64)
    p_ref, a_ref, cnt = oracle.gravity_walk(mesh, rho, ewald="table", table=tab)
    _, p64, a64, st = run_gravity(mesh, rho, precision="fp64", ewald_n=64)
    assert e_a(a64, a_ref).max() < 1e-9
    np.testing.assert_allclose(p64, p_ref, rtol=1e-9, atol=1e-9 * np.abs(p_ref).max())
    assert st["interactions"] == cnt["interactions"]


@pytest.mark.parametrize("bc,box", BOXES)
def test_fp32_walk_against_exact_series(oracle, bc, box):
    mesh, rho = _mesh(bc, box, n=16, seed=1)
    tg = I.sample_cells(mesh.ncell, 200, seed=2)
    p_ref, a_ref, _ = oracle.gravity_walk(mesh, rho, tg, ewald="series")
    _, p32, a32, _ = run_gravity(mesh, rho, precision="fp32", ewald_n=64 if bc != (1, 0, 0) else 32)
    e = e_a(a32[tg], a_ref)
    assert np.median(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2, (np.median(e), e.max())
    dp = (p32[tg] - p32[tg].mean()) - (p_ref - p_ref.mean())
    assert np.median(np.abs(dp)) < 1e-3 * np.abs(p_ref).max()


def test_uniform_periodic_box_zero_force_and_zero_mean(oracle):
    """Uniform density, fully periodic: the exact field vanishes and the exact potential is flat;
    the BH walk leaves only its monopole error, which must equal the oracle's same-MAC walk."""
    mesh = I.uniform_mesh(32, bc=(1, 1, 1))
    rho = np.ones((mesh.nleaf, 8, 8, 8))
    _, p, a, _ = run_gravity(mesh, rho, precision="fp32", zero_mean=True)
    assert np.abs(a).max() < 1e-3 * (4 * np.pi / 3)
    assert abs(p.mean()) < 1e-6
    tg = I.sample_cells(mesh.ncell, 64, seed=3)
    tab = oracle.ewald_table((1, 1, 1), (1.0, 1.0, 1.0), n=64)
    pr, ar, _ = oracle.gravity_walk(mesh, rho, tg, ewald="table", table=tab)
    dp = (p[tg] - p[tg].mean()) - (pr - pr.mean())
    assert np.abs(dp).max() < 1e-5
    np.testing.assert_allclose(a[tg], ar, atol=1e-5)


def test_jeans_wave_periodic(oracle):
    mesh = I.uniform_mesh(32, bc=(1, 1, 1))
    x = mesh.cell_centres()
    k = 2 * np.pi
    rho = 1.0 + 0.5 * np.cos(k * x[..., 0])
    _, p, a, _ = run_gravity(mesh, rho, precision="fp32", zero_mean=True)
    ax = -4 * np.pi * 0.5 * np.sin(k * x.reshape(-1, 3)[:, 0]) / k
    assert np.abs(a[:, 0] - ax).max() < 0.02 * np.abs(ax).max()
