"""Pins of the oracle's l_q-quantity column maps and the pixel-averaged shielding quantities
(Sec. 2.3): a quantity proportional to the density maps to the proportional map, maps are linear in
the quantity, an opened-everywhere walk conserves each quantity's mass exactly (brute force over the
cells), and the pixel averages reduce to their per-direction functions for uniform maps, mix with
the pixel weights for non-uniform ones, and reproduce any bilinear CO table exactly.  The H2
self-shielding function itself is typed from its published source (parity unpinned: the paper
prints no values of it)."""
import numpy as np

from paper_1708_06142_gb300 import inputs as I


def _mesh():
    mesh, rho = I.sphere_32(seed=0, ncell_axis=16)
    rng = np.random.default_rng(4)
    x, y, z = mesh.cell_centres().reshape(-1, 3).T
    q1 = rho.reshape(-1) * (0.5 + 0.5 * np.tanh((z - 0.5) / 0.1))            # an H2-like fraction
    q2 = rho.reshape(-1) * 1e-4 * rng.uniform(0, 1, mesh.ncell)               # a CO-like fraction
    return mesh, rho, q1, q2


def test_proportional_and_linear_quantities(oracle):
    mesh, rho, q1, q2 = _mesh()
    tg = I.sample_cells(mesh.ncell, 60, seed=2)
    cols, _ = oracle.column_walk(mesh, rho, tg, quantities=np.stack([0.3 * rho.reshape(-1), q1]))
    assert cols.shape == (60, 3, 48)
    np.testing.assert_allclose(cols[:, 1], 0.3 * cols[:, 0], rtol=1e-12)
    a, _ = oracle.column_walk(mesh, rho, tg, quantities=np.stack([q1, q2]))
    b, _ = oracle.column_walk(mesh, rho, tg, quantities=(q1 + q2)[None])
    np.testing.assert_allclose(b[:, 1], a[:, 1] + a[:, 2], rtol=1e-12, atol=1e-300)
    # the total-mass map is the plain column walk's
    c0, _ = oracle.column_walk(mesh, rho, tg)
    np.testing.assert_array_equal(a[:, 0], c0)


def test_quantity_mass_conservation_brute_force(oracle):
    # theta -> 0 opens every node: each cell is mapped on its own, and with weights summing to one
    # sum_i N_q,i Omega = sum_{c' != c} m_q(c') / |d|^2 + 4 pi rho_q(c) dx / 2
    mesh, rho, q1, q2 = _mesh()
    tg = I.sample_cells(mesh.ncell, 12, seed=5)
    cols, _ = oracle.column_walk(mesh, rho, tg, theta=1e-6, quantities=np.stack([q1, q2]))
    cen = mesh.cell_centres().reshape(-1, 3)
    dv = np.repeat(mesh.cell_volume(), 512)
    dx = np.repeat(mesh.size[mesh.leaves][:, 0] / 8, 512)
    omega = 4 * np.pi / 48
    for t, c in enumerate(tg):
        d2 = ((cen - cen[c]) ** 2).sum(1)
        d2[c] = np.inf
        for k, q in enumerate((q1, q2)):
            want = (q * dv / d2).sum() + 4 * np.pi * q[c] * dx[c] / 2
            assert cols[t, 1 + k].sum() * omega == pytest_approx(want)


def pytest_approx(v):
    import pytest
    return pytest.approx(v, rel=1e-11)


def test_shielding_averages(oracle):
    rng = np.random.default_rng(1)
    npix = 48
    # uniform maps: the averages are the per-direction functions themselves
    n_tot, n_h2, n_co = 2.0, 3e15, 1e14
    cols = np.stack([np.full(npix, n_tot), np.full(npix, n_h2), np.full(npix, n_co)])[None]
    tab = rng.uniform(0.1, 1.0, (5, 7))
    s = oracle.column_shielding(cols, k_av=1.0, k_h2=1.0, b5=2.0, co_table=tab, lg_co=(12.0, 16.0),
                                lg_h2=(14.0, 20.0))[0]
    assert abs(s[0] - n_tot) < 1e-12
    assert abs(s[1] - oracle.h2_self_shielding(n_h2, 2.0)) < 1e-15
    # one pixel blocked: the pixel weights 1/N_PIX
    cols2 = cols.copy()
    cols2[0, 1, 0] = 1e25
    s2 = oracle.column_shielding(cols2, b5=2.0)[0]
    want = (47 * oracle.h2_self_shielding(n_h2, 2.0) + oracle.h2_self_shielding(1e25, 2.0)) / 48
    assert abs(s2[1] - want) < 1e-15
    assert s2[2] == 1.0                                    # no CO table: no CO shielding
    # a table linear in (log N_CO, log N_H2) is reproduced exactly by the bilinear lookup
    gco, gh2 = np.linspace(12, 16, 5), np.linspace(14, 20, 7)
    lin = 0.1 + 0.05 * (gco[:, None] - 12) + 0.02 * (gh2[None, :] - 14)
    lc, lh = rng.uniform(12, 16, npix), rng.uniform(14, 20, npix)
    cols3 = np.stack([np.zeros(npix), 10.0 ** lh, 10.0 ** lc])[None]
    s3 = oracle.column_shielding(cols3, co_table=lin, lg_co=(12.0, 16.0), lg_h2=(14.0, 20.0))[0]
    assert abs(s3[2] - np.mean(0.1 + 0.05 * (lc - 12) + 0.02 * (lh - 14))) < 1e-12
    assert s3[0] == 0.0
    # the H2 factor falls with the column and is 0.965 + 0.035 e^-8.5e-4 for no column
    f = oracle.h2_self_shielding(np.logspace(10, 24, 50), 3.0)
    assert np.all(np.diff(f) < 0)
    assert abs(oracle.h2_self_shielding(0.0) - (0.965 + 0.035 * np.exp(-8.5e-4))) < 1e-15
