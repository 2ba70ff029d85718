"""GPU parity of the node-ray table and the column-density walk against the FP64 oracle."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(mesh, rho, **kw):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    p = ts.column_params(**kw)
    npix = 12 * p.n_side ** 2
    cols = torch.empty(mesh.ncell, npix, dtype=torch.float32, device="cuda")
    ts.column_walk(cols, p)
    ts.sync()
    return ts, cols.cpu().numpy().astype(np.float64)


def test_noderay_table_matches_oracle(oracle):
    mesh, rho = I.turbulent_periodic(seed=3, n=16)
    ts, _ = _run(mesh, rho, n_side=2)
    t = ts.noderay_table()
    ref = oracle.noderay_table(2)
    assert t.shape == ref.shape
    # weights are counts / nsub^3; a sub-cube centre exactly on a pixel edge may land differently
    diff = np.abs(t - ref)
    assert (diff > 1e-12).mean() < 1e-4 and diff.max() <= 2.0 / 512 + 1e-12


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_column_walk_matches_oracle(oracle, bc):
    mesh = I.uniform_mesh(32, bc=bc)
    rng = np.random.default_rng(7)
    rho = np.exp(rng.standard_normal((mesh.nleaf, 8, 8, 8)))
    tg = I.sample_cells(mesh.ncell, 300, seed=1)
    ref, cnt = oracle.column_walk(mesh, rho, tg, nside=2, theta=0.5)
    _, cols = _run(mesh, rho, n_side=2, theta=0.5)
    rel = np.abs(cols[tg] - ref) / ref
    # bin choices are taken in FP32 on the device and FP64 in the oracle: a rare near-edge node
    # lands in a neighbouring table bin, so the tolerance is on the median and the 99th percentile
    assert np.median(rel) < 1e-4 and np.quantile(rel, 0.99) < 1e-2, (np.median(rel), np.quantile(rel, 0.99))


def test_uniform_sphere_centre_column():
    mesh = I.uniform_mesh(64)
    c = np.array([32.5, 32.5, 32.5]) / 64
    x = mesh.cell_centres()
    r = np.sqrt(((x - c) ** 2).sum(-1))
    rho = np.where(r < 0.3, 1.0, 0.0)
    _, cols = _run(mesh, rho, n_side=2, theta=0.5)
    t = int(np.argmin(r.reshape(-1)))
    assert abs(cols[t].mean() / 0.3 - 1) < 0.03
    assert np.abs(cols[t] / 0.3 - 1).max() < 0.2
