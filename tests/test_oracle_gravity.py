"""Pins for the oracle's gravity walk and N^2 reference (Secs. 2.1, 2.2.1-2.2.2, 3).

- theta -> 0 opens every node, so the tree walk must equal the direct N^2 sum.
- closed forms: potential outside a uniform sphere (-M/r up to its small cubic-lattice
  hexadecapole), Gauss's law inside it, the Jeans sine wave in a periodic box (Sec. 3.1.2),
  a uniform periodic box (no force), and Gauss's law for plane layers with 2P1I BCs.
"""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I


def _ea(a, aref):
    return np.linalg.norm(a - aref, axis=1) / np.linalg.norm(aref, axis=1).max()


def test_theta_zero_equals_direct_sum_amr(oracle):
    mesh, rho = I.plummer_amr(seed=7, max_level=4)
    tg = I.sample_cells(mesh.ncell, 200, seed=3)
    p0, a0, c0 = oracle.gravity_walk(mesh, rho, tg, theta=0.0)
    pd, ad = oracle.direct_sum(mesh, rho, tg)
    assert c0["interactions"] == tg.size * (mesh.ncell - 1)
    np.testing.assert_allclose(p0, pd, rtol=1e-12)
    assert np.abs(a0 - ad).max() <= 1e-12 * np.abs(ad).max()


def test_ape_zero_limit_equals_direct_sum(oracle):
    mesh, rho = I.sphere_32(seed=4)
    tg = I.sample_cells(mesh.ncell, 100, seed=4)
    p0, a0, _ = oracle.gravity_walk(mesh, rho, tg, mac="ape", a_lim=0.0)
    pd, ad = oracle.direct_sum(mesh, rho, tg)
    np.testing.assert_allclose(p0, pd, rtol=1e-12)
    assert np.abs(a0 - ad).max() <= 1e-12 * np.abs(ad).max()


def test_bh_error_decreases_with_theta(oracle):
    mesh, rho = I.sphere_32(seed=0)
    tg = I.sample_cells(mesh.ncell, 400, seed=9)
    pd, ad = oracle.direct_sum(mesh, rho, tg)
    med = []
    for th in (1.0, 0.5, 0.25):
        _, a, _ = oracle.gravity_walk(mesh, rho, tg, theta=th)
        med.append(np.median(_ea(a, ad)))
    assert med[0] > med[1] > med[2]
    assert med[1] < 2e-3          # BH theta = 0.5 is accurate to ~1e-3 (Sec. 3 tables)


def test_uniform_sphere_outside_potential_and_inside_gauss(oracle):
    mesh = I.uniform_mesh(32)
    c = np.array([16.5, 16.5, 16.5]) / 32
    x = mesh.cell_centres()
    r = np.sqrt(((x - c) ** 2).sum(-1))
    R = 0.3
    rho = np.where(r < R, 1.0, 0.0)
    M = (rho * mesh.cell_volume()[:, None, None, None]).sum()
    flat_r = r.reshape(-1)
    far = np.nonzero(flat_r > 0.75)[0]
    pd, ad = oracle.direct_sum(mesh, rho, far)
    np.testing.assert_allclose(pd, -M / flat_r[far], rtol=2e-3)
    inner = np.nonzero((flat_r > 0.1) & (flat_r < 0.2))[0][::7]
    pd, ad = oracle.direct_sum(mesh, rho, inner)
    xr = x.reshape(-1, 3)[inner] - c
    a_exact = -(4.0 / 3.0) * np.pi * 1.0 * xr
    assert np.median(np.linalg.norm(ad - a_exact, axis=1) / np.linalg.norm(a_exact, axis=1)) < 0.03


def test_uniform_periodic_box_has_no_force(oracle):
    mesh = I.uniform_mesh(8, bc=(1, 1, 1))
    rho = np.ones((mesh.nleaf, 8, 8, 8))
    tg = np.arange(0, 512, 37)
    pd, ad = oracle.direct_sum(mesh, rho, tg)
    assert np.abs(ad).max() < 1e-10
    assert np.ptp(pd) < 1e-10


def test_jeans_sine_wave_periodic(oracle):
    # rho = 1 + 0.5 cos(k x): a_x = -4 pi G rho1 sin(k x) / k  (Sec. 3.1.2)
    n = 16
    mesh = I.uniform_mesh(n, bc=(1, 1, 1))
    x = mesh.cell_centres()
    k = 2 * np.pi
    rho = 1.0 + 0.5 * np.cos(k * x[..., 0])
    xf = x.reshape(-1, 3)
    tg = np.nonzero((np.abs(xf[:, 1] - 0.5 / n) < 1e-12) & (np.abs(xf[:, 2] - 0.5 / n) < 1e-12))[0]
    pd, ad = oracle.direct_sum(mesh, rho, tg)
    ax = -4 * np.pi * 0.5 * np.sin(k * xf[tg, 0]) / k
    assert np.abs(ad[:, 0] - ax).max() < 0.02 * np.abs(ax).max()
    assert np.abs(ad[:, 1:]).max() < 1e-9


def test_planar_layers_gauss_law_2p1i(oracle):
    # density depending on z only, x,y periodic: a_z = -2 pi G (Sigma_below - Sigma_above)
    mesh = I.uniform_mesh(8, box=(1.0, 1.0, 1.0), bc=(1, 1, 0))
    x = mesh.cell_centres()
    rho = 1.0 + np.exp(-((x[..., 2] - 0.4) / 0.2) ** 2)
    tg = np.arange(0, 512, 9)
    pd, ad = oracle.direct_sum(mesh, rho, tg)
    z = x.reshape(-1, 3)[:, 2]
    sig = (rho * mesh.cell_volume()[:, None, None, None]).reshape(-1)  # area Lx*Ly = 1
    az = np.array([-2 * np.pi * (sig[z < z[t] - 1e-12].sum() - sig[z > z[t] + 1e-12].sum()) for t in tg])
    assert np.abs(ad[:, 2] - az).max() < 1e-2 * np.abs(az).max()
    assert np.abs(ad[:, :2]).max() < 1e-2 * np.abs(az).max()


def test_ewald_table_walk_close_to_series_walk(oracle):
    mesh, rho = I.uniform_mesh(16, box=(1.0, 1.0, 2.0), bc=(1, 1, 0)), None
    rng = np.random.default_rng(0)
    rho = np.exp(rng.standard_normal((mesh.nleaf, 8, 8, 8)) * 0.5)
    tg = I.sample_cells(mesh.ncell, 60, seed=1)
    tab = oracle.ewald_table(mesh.bc, mesh.domain_size, n=64)
    ps, as_, _ = oracle.gravity_walk(mesh, rho, tg, ewald="series")
    pt, at, _ = oracle.gravity_walk(mesh, rho, tg, ewald="table", table=tab)
    assert np.median(_ea(at, as_)) < 1e-4
    dp = (pt - pt.mean()) - (ps - ps.mean())
    assert np.abs(dp).max() < 1e-4 * np.abs(ps).max()
