"""Pins for the oracle's gravity walk and N^2 reference (Secs. 2.1, 2.2.1-2.2.2, 3).

- theta -> 0 opens every node, so the tree walk must equal the direct N^2 sum.
- on one 8^3 block, a brute-force walk over the cube geometry (moments by numpy sums) gives the
  same interactions and potentials for any theta and eta_SB (the safe box of Sec. 2.1), with the
  closed-form count of 21 interactions per target for theta -> infinity, eta_SB = 1.2.
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


@pytest.mark.parametrize("mac,theta,eta", [("bh", 1e6, 1.2), ("bh", 1e6, 0.0), ("bh", 1e6, 2.0), ("bh", 1e6, 2.6),
                                           ("bh", 0.7, 1.2), ("bh", 0.4, 2.0), ("ape", 1e-3, 1.2), ("ape", 3e-2, 0.0)])
def test_walk_on_one_block_equals_brute_force(oracle, mac, theta, eta):
    """One 8^3 leaf-block: its tree is the block node, 8 level-1 nodes of 4^3 cells, 64 level-2
    nodes of 2^3 cells and the cells.  Brute force over that geometry (node moments by numpy sums of
    the cells inside each cube): a node is accepted when the BH MAC passes (longest edge / distance to
    the centre of mass < theta) and the target lies outside the eta_SB box about the node's
    geometric centre (Sec. 2.1), else opened; an opened level-2 node's cells are accepted, the
    target's own cell excluded.  With mac = "ape", theta is the absolute limit a_lim of eq. ape
    (accept when G M h^2 / d^4 < a_lim, G = 1).  Interaction counts must agree exactly, potentials
    to rounding.
    For theta -> infinity and eta = 1.2 every target makes 21 interactions (7 + 7 + 7 siblings of
    its own level-1 node, level-2 node and cell); for eta = 0 the block node is accepted alone."""
    mesh = I.uniform_mesh(8)
    rng = np.random.default_rng(5)
    rho = rng.random((1, 8, 8, 8)) + 0.5
    dx = 1.0 / 8
    idx = np.stack(np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij"), -1)   # [k, j, i, (k, j, i)]
    x = (idx[..., ::-1] + 0.5) * dx                     # cell centres (x, y, z), natural order [k, j, i]
    m = rho[0] * dx ** 3
    tg = I.sample_cells(512, 48, seed=2)
    if mac == "bh":
        pot_ref, _, cnt = oracle.gravity_walk(mesh, rho, tg, theta=theta, safe_box=eta)
    else:
        pot_ref, _, cnt = oracle.gravity_walk(mesh, rho, tg, mac="ape", a_lim=theta, safe_box=eta)

    def node(lo, size):
        sel = np.all((x >= lo) & (x < lo + size), axis=-1)
        mm = m[sel].sum()
        return mm, (m[sel][:, None] * x[sel]).sum(0) / mm

    def visit(t, lo, size, level):
        """(interactions, potential) of the subtree of the cube [lo, lo + size)"""
        xt = x.reshape(-1, 3)[t]
        mm, com = node(lo, size)
        d = np.linalg.norm(xt - com)
        inside = np.all(np.abs(xt - (lo + size / 2)) <= eta * size / 2)
        mac_ok = size / d < theta if mac == "bh" else mm * size ** 2 / d ** 4 < theta
        if d > 0 and mac_ok and not inside:
            return 1, -mm / d
        if level == 2:                                  # open a level-2 node: its 8 cells
            n, p = 0, 0.0
            for o in range(8):
                c = lo + dx * np.array([o & 1, (o >> 1) & 1, o >> 2])
                cid = int(np.rint(c[2] / dx)) * 64 + int(np.rint(c[1] / dx)) * 8 + int(np.rint(c[0] / dx))
                if cid != t:
                    n += 1
                    p -= m.reshape(-1)[cid] / np.linalg.norm(xt - (c + dx / 2))
            return n, p
        n, p = 0, 0.0
        for o in range(8):
            n1, p1 = visit(t, lo + size / 2 * np.array([o & 1, (o >> 1) & 1, o >> 2]), size / 2, level + 1)
            n, p = n + n1, p + p1
        return n, p

    res = [visit(int(t), np.zeros(3), 1.0, 0) for t in tg]
    assert sum(r[0] for r in res) == cnt["interactions"]
    np.testing.assert_allclose([r[1] for r in res], pot_ref, rtol=1e-12)
    if mac == "bh" and theta > 1e3 and eta == 1.2:
        assert cnt["interactions"] == 21 * tg.size
    if mac == "bh" and eta == 0.0:
        assert cnt["interactions"] == tg.size
