"""Pins for the oracle's tree build (Sec. 2.1: bottom-up sums of mass and centre of mass).

Each node's moments are recomputed here by brute force over the cells it covers (numpy slicing
of the cell arrays, a different route from the oracle's index arithmetic), on small meshes.
"""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I


def _cell_mass(mesh, rho):
    return rho * mesh.cell_volume()[:, None, None, None]


def test_block_tree_nodes_brute_force(oracle):
    mesh, rho = I.plummer_amr(seed=5, max_level=4)
    T = oracle.tree_build(mesh, rho)
    m = _cell_mass(mesh, rho)
    x = mesh.cell_centres()
    nl = mesh.nleaf
    # level-2 nodes: 2x2x2 cells, index p = px + 4 py + 16 pz
    m2 = m.reshape(nl, 4, 2, 4, 2, 4, 2).sum(axis=(2, 4, 6)).reshape(nl, 64)
    mx2 = (m[..., None] * x).reshape(nl, 4, 2, 4, 2, 4, 2, 3).sum(axis=(2, 4, 6)).reshape(nl, 64, 3)
    np.testing.assert_allclose(T["n2_mass"], m2, rtol=1e-13)
    np.testing.assert_allclose(T["n2_com"], mx2 / m2[..., None], rtol=1e-13)
    # level-1 nodes: 4x4x4 cells, index q = qx + 2 qy + 4 qz
    m1 = m.reshape(nl, 2, 4, 2, 4, 2, 4).sum(axis=(2, 4, 6)).reshape(nl, 8)
    mx1 = (m[..., None] * x).reshape(nl, 2, 4, 2, 4, 2, 4, 3).sum(axis=(2, 4, 6)).reshape(nl, 8, 3)
    np.testing.assert_allclose(T["n1_mass"], m1, rtol=1e-13)
    np.testing.assert_allclose(T["n1_com"], mx1 / m1[..., None], rtol=1e-13)


def test_amr_block_moments_brute_force(oracle):
    mesh, rho = I.plummer_amr(seed=6, max_level=4)
    T = oracle.tree_build(mesh, rho)
    m = _cell_mass(mesh, rho).reshape(-1)
    x = mesh.cell_centres().reshape(-1, 3)
    for b in range(mesh.nblocks):
        lo, hi = mesh.lo[b], mesh.lo[b] + mesh.size[b]
        inside = np.all((x > lo) & (x < hi), axis=1)
        M = m[inside].sum()
        assert T["block_mass"][b] == pytest.approx(M, rel=1e-12)
        np.testing.assert_allclose(T["block_com"][b], (m[inside, None] * x[inside]).sum(0) / M, rtol=1e-12)


def test_root_mass_and_symmetric_centre(oracle):
    # a density symmetric under reflection through the box centre has its CoM at the centre
    mesh = I.uniform_mesh(32)
    r = mesh.cell_centres() - 0.5
    rho = np.exp(-(r ** 2).sum(-1) / 0.02) + 0.1 * np.cos(2 * np.pi * r[..., 0]) ** 2
    T = oracle.tree_build(mesh, rho)
    assert T["block_mass"][0] == pytest.approx((rho * mesh.cell_volume()[:, None, None, None]).sum(), rel=1e-14)
    np.testing.assert_allclose(T["block_com"][0], [0.5, 0.5, 0.5], atol=1e-14)


def test_zero_mass_node_centre_is_geometric(oracle):
    mesh = I.uniform_mesh(16)
    rho = np.zeros((mesh.nleaf, 8, 8, 8))
    rho[0] = 1.0
    T = oracle.tree_build(mesh, rho)
    lf = mesh.leaves
    for n in range(1, mesh.nleaf):
        b = lf[n]
        assert T["block_mass"][b] == 0.0
        np.testing.assert_allclose(T["block_com"][b], mesh.lo[b] + 0.5 * mesh.size[b])
