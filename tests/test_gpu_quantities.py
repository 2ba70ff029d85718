"""l_q = 3 column maps (total, H2, CO) and the pixel-averaged shielding quantities on the GPU
(Sec. 2.3) against the FP64 oracle."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _fields(mesh, seed=3):
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.standard_normal((mesh.nleaf, 8, 8, 8))).reshape(-1)
    z = mesh.cell_centres().reshape(-1, 3)[:, 2]
    h2 = rho * (0.5 + 0.5 * np.tanh((z - 0.5) / 0.1))
    co = rho * 1e-4 * rng.uniform(0.0, 1.0, mesh.ncell)
    return rho, np.stack([h2, co])


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_quantity_maps_match_oracle(oracle, bc):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    mesh = I.uniform_mesh(32, bc=bc)
    rho, q = _fields(mesh)
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho).cuda())
    p = ts.column_params(n_side=2, theta=0.5)
    plain = torch.empty(mesh.ncell, 48, device="cuda")
    ts.column_walk(plain, p)
    ts.column_quantities(torch.from_numpy(q).cuda())
    cols = torch.empty(mesh.ncell, 3, 48, device="cuda")
    ts.column_walk(cols, p)
    ts.sync()
    cols = cols.cpu().numpy().astype(np.float64)
    # the total map is the plain walk's
    np.testing.assert_allclose(cols[:, 0], plain.cpu().numpy(), rtol=1e-6)
    tg = I.sample_cells(mesh.ncell, 200, seed=1)
    ref, _ = oracle.column_walk(mesh, rho.reshape(mesh.nleaf, 8, 8, 8), tg, nside=2, theta=0.5, quantities=q)
    for k in range(3):
        got, want = cols[tg, k], ref[:, k]
        # per-cell totals are independent of table-bin choices (see test_gpu_column)
        assert np.abs(got.sum(1) - want.sum(1)).max() <= 1e-5 * want.sum(1).max(), k
        rel = np.abs(got - want) / want
        off = rel > 1e-4
        assert np.median(rel) < 1e-5 and off.mean() < 0.01, (k, np.median(rel), off.mean())
    # a new tree build drops the quantities
    ts.tree_build(None, torch.from_numpy(rho).cuda())
    ts.column_walk(plain, p)
    ts.sync()


def test_shielding_matches_oracle(oracle):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    rng = np.random.default_rng(2)
    n, npix = 1037, 48
    cols = np.stack([np.exp(rng.normal(-1.0, 1.5, (n, npix))),              # total, in A_V units
                     10.0 ** rng.uniform(12.0, 22.0, (n, npix)),             # N_H2 [cm^-2]
                     10.0 ** rng.uniform(10.0, 19.0, (n, npix))], 1).astype(np.float32)
    tab = rng.uniform(0.01, 1.0, (9, 11))
    kw = dict(k_av=0.7, k_h2=1.0, b5=2.0, k_co=1.0, co_table=tab, lg_co=(11.0, 18.0), lg_h2=(13.0, 21.0))
    out = torch.empty(n, 3, device="cuda")
    ts = TreeSolver(0)
    ts.column_shielding(torch.from_numpy(cols).cuda(), out, **kw)
    ts.sync()
    got = out.cpu().numpy().astype(np.float64)
    ref = oracle.column_shielding(cols.astype(np.float64), **kw)
    np.testing.assert_allclose(got[:, 0], ref[:, 0], rtol=2e-5, atol=2e-6)
    np.testing.assert_allclose(got[:, 1], ref[:, 1], rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(got[:, 2], ref[:, 2], rtol=1e-4, atol=1e-6)
    # without a CO table the CO factor is 1
    kw.pop("co_table")
    ts.column_shielding(torch.from_numpy(cols).cuda(), out, **kw)
    ts.sync()
    assert np.all(out.cpu().numpy()[:, 2] == 1.0)


def test_quantity_errors():
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver, TSError
    mesh = I.uniform_mesh(16)
    ts = TreeSolver(0)
    ts.ncell = mesh.ncell     # the binding learns ncell from a build; the library has no tree yet
    with pytest.raises(TSError) as e:
        ts.column_quantities(torch.zeros(1, mesh.ncell, dtype=torch.float64, device="cuda"))
    assert e.value.status == 5
    ts.tree_build(mesh, torch.ones(mesh.ncell, dtype=torch.float64, device="cuda"))
    with pytest.raises(TSError) as e:
        ts.column_quantities(torch.zeros(3, mesh.ncell, dtype=torch.float64, device="cuda"))
    assert e.value.status == 1
    ts.column_quantities(torch.zeros(2, mesh.ncell, dtype=torch.float64, device="cuda"))
    with pytest.raises(TSError) as e:        # 3 maps of 192 pixels do not fit in shared memory
        ts.column_walk(torch.empty(mesh.ncell, 3, 192, device="cuda"), ts.column_params(n_side=4))
    assert e.value.status == 2
