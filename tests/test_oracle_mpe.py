"""Pins for the oracle's MPE MAC (Sec. 2.2.1, eq. mpe with p = 1).

- B_p = sum_i m_i |r_i - r_a|^p of every level-2, level-1 and block node against numpy sums over the
  node's cells, and against the closed form of a uniform node (all cells at their own distances).
- the bound: for an accepted node the monopole's acceleration error is at most Delta a_max
  (SW94); checked node by node against the exact sum over the node's cells, for targets outside
  b_max, so a wrong exponent or coefficient in the formula fails it.
- the walk: its total error is at most (accepted interactions) x a_lim per target, a_lim -> 0
  reproduces the N^2 sum, and a larger a_lim accepts fewer, larger nodes.
"""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I


def _mesh(seed=0):
    mesh = I.build_mesh(lambda lvl, lo, size: lvl < 2 or (lvl < 3 and lo[0] < 0.4 and lo[1] < 0.6))
    rng = np.random.default_rng(seed)
    rho = np.exp(0.8 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))
    return mesh, rho


def _cells(mesh, rho):
    x = mesh.cell_centres().reshape(mesh.nleaf, 8, 8, 8, 3)
    m = rho * mesh.cell_volume()[:, None, None, None]
    return x, m


def test_bmoments_match_cell_sums(oracle):
    mesh, rho = _mesh()
    B = oracle.tree_bmoments(mesh, rho)
    mom = oracle.tree_build(mesh, rho)
    x, m = _cells(mesh, rho)
    for n in range(mesh.nleaf):
        for p in range(64):                                   # level-2 node p = px + 4 py + 16 pz
            px, py, pz = p & 3, (p >> 2) & 3, p >> 4
            sl = (n, slice(2 * pz, 2 * pz + 2), slice(2 * py, 2 * py + 2), slice(2 * px, 2 * px + 2))
            d = np.linalg.norm(x[sl] - mom["n2_com"][n, p], axis=-1)
            np.testing.assert_allclose(B["n2"][n, p], [(m[sl] * d ** 2).sum(), (m[sl] * d ** 3).sum()], rtol=1e-12)
        for q in range(8):
            qx, qy, qz = q & 1, (q >> 1) & 1, q >> 2
            sl = (n, slice(4 * qz, 4 * qz + 4), slice(4 * qy, 4 * qy + 4), slice(4 * qx, 4 * qx + 4))
            d = np.linalg.norm(x[sl] - mom["n1_com"][n, q], axis=-1)
            np.testing.assert_allclose(B["n1"][n, q], [(m[sl] * d ** 2).sum(), (m[sl] * d ** 3).sum()], rtol=1e-12)
    # every block (leaf or not): all cells below it
    leaves = mesh.leaves
    lo, hi = mesh.lo, mesh.lo + mesh.size
    for b in range(mesh.nblocks):
        inside = np.all((mesh.lo[leaves] >= lo[b] - 1e-12) & (mesh.lo[leaves] < hi[b] - 1e-12), axis=1)
        d = np.linalg.norm(x[inside] - mom["block_com"][b], axis=-1)
        np.testing.assert_allclose(B["block"][b], [(m[inside] * d ** 2).sum(), (m[inside] * d ** 3).sum()],
                                   rtol=1e-12)


def test_bmoments_uniform_closed_form(oracle):
    mesh = I.uniform_mesh(8)
    rho = np.full((1, 8, 8, 8), 2.0)
    B = oracle.tree_bmoments(mesh, rho)
    dx = 1.0 / 8
    mc = 2.0 * dx ** 3
    # level-2 node: 8 cells at distance sqrt(3) dx / 2 from its centre
    r = np.sqrt(3) * dx / 2
    np.testing.assert_allclose(B["n2"][0, 0], [8 * mc * r ** 2, 8 * mc * r ** 3], rtol=1e-13)
    # level-1 node: 64 cells at offsets (+-1/2, +-3/2) dx per axis
    o = np.array([-1.5, -0.5, 0.5, 1.5]) * dx
    d2 = o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2
    np.testing.assert_allclose(B["n1"][0, 0], [mc * d2.sum(), mc * (d2 ** 1.5).sum()], rtol=1e-13)


def test_mpe_bound_holds_node_by_node(oracle):
    mesh, rho = _mesh(1)
    B = oracle.tree_bmoments(mesh, rho)
    mom = oracle.tree_build(mesh, rho)
    x, m = _cells(mesh, rho)
    rng = np.random.default_rng(2)
    checked = 0
    for n in range(mesh.nleaf):
        b = mesh.leaves[n]
        for q in range(8):
            qx, qy, qz = q & 1, (q >> 1) & 1, q >> 2
            sl = (n, slice(4 * qz, 4 * qz + 4), slice(4 * qy, 4 * qy + 4), slice(4 * qx, 4 * qx + 4))
            ra, M = mom["n1_com"][n, q], mom["n1_mass"][n, q]
            half = mesh.size[b] / 4
            cen = mesh.lo[b] + (np.array([qx, qy, qz]) + 0.5) * 2 * half
            bmax = np.linalg.norm(half + np.abs(ra - cen))
            B2, B3 = B["n1"][n, q]
            for _ in range(3):
                u = rng.standard_normal(3)
                r = ra + u / np.linalg.norm(u) * bmax * rng.uniform(1.2, 6.0)
                d = np.linalg.norm(r - ra)
                dv = r - x[sl].reshape(-1, 3)
                exact = -(m[sl].reshape(-1, 1) * dv / np.linalg.norm(dv, axis=1)[:, None] ** 3).sum(0)
                mono = -M * (r - ra) / d ** 3
                bound = 1.0 / d ** 2 / (1 - bmax / d) ** 2 * (3 * B2 / d ** 2 - 2 * B3 / d ** 3)
                assert np.linalg.norm(exact - mono) <= bound * (1 + 1e-12)
                checked += 1
    assert checked > 100


def test_mpe_walk_error_within_summed_bounds(oracle):
    mesh, rho = _mesh(3)
    tg = I.sample_cells(mesh.ncell, 24, seed=4)
    _, a_dir = oracle.direct_sum(mesh, rho, tg)
    amax = np.linalg.norm(a_dir, axis=1).max()
    for a_lim in (1e-2 * amax, 1e-3 * amax):
        for t in tg:
            _, a, cnt = oracle.gravity_walk(mesh, rho, np.array([t]), mac="mpe", a_lim=a_lim)
            err = np.linalg.norm(a[0] - a_dir[tg == t][0])
            assert err <= cnt["interactions"] * a_lim
    # a_lim -> 0 opens every node down to the cells: the N^2 sum
    _, a0, _ = oracle.gravity_walk(mesh, rho, tg, mac="mpe", a_lim=1e-300)
    np.testing.assert_allclose(a0, a_dir, rtol=1e-11, atol=1e-12 * amax)
    # looser limits accept more distant approximations: fewer interactions
    counts = [oracle.gravity_walk(mesh, rho, tg, mac="mpe", a_lim=f * amax)[2]["interactions"]
              for f in (1e-4, 1e-3, 1e-2)]
    assert counts[0] > counts[1] > counts[2]


def test_mpe_bound_is_attained_for_a_collinear_pair(oracle):
    # two equal masses on the line of sight: the monopole error is m [(d - s)^-2 + (d + s)^-2 - 2 d^-2]
    # ~ 6 m s^2 / d^4, which the bound's leading term 3 B2 / d^4 (B2 = 2 m s^2) reaches as d grows,
    # so the bound must hold and be tight (a coefficient or exponent error breaks one of the two)
    mesh = I.uniform_mesh(8)
    rho = np.zeros((1, 8, 8, 8))
    rho[0, 0, 0, 0] = rho[0, 1, 1, 1] = 1.0                 # cells (0,0,0) and (1,1,1) of level-2 node 0
    B = oracle.tree_bmoments(mesh, rho)
    mom = oracle.tree_build(mesh, rho)
    ra, M = mom["n2_com"][0, 0], mom["n2_mass"][0, 0]
    B2, B3 = B["n2"][0, 0]
    half, cen = np.full(3, 1 / 8), np.full(3, 1 / 8)           # node [0, 1/4]^3
    bmax = np.linalg.norm(half + np.abs(ra - cen))
    assert bmax == pytest.approx(np.sqrt(3) / 8)
    x, m = _cells(mesh, rho)
    u = np.ones(3) / np.sqrt(3)
    ratios = []
    for f in (1.5, 3.0, 10.0, 50.0):
        r = ra + u * bmax * f
        d = np.linalg.norm(r - ra)
        dv = r - x.reshape(-1, 3)
        w = m.reshape(-1) > 0
        exact = -(m.reshape(-1)[w, None] * dv[w] / np.linalg.norm(dv[w], axis=1)[:, None] ** 3).sum(0)
        err = np.linalg.norm(exact + M * (r - ra) / d ** 3)
        bound = 1.0 / d ** 2 / (1 - bmax / d) ** 2 * (3 * B2 / d ** 2 - 2 * B3 / d ** 3)
        ratios.append(err / bound)
    assert max(ratios) <= 1.0
    assert ratios[-1] > 0.85, ratios


def test_mpe_walk_decides_at_the_bound(oracle):
    # one leaf-block; the target cell (7,7,7) and level-1 node 0 ([0, 1/2]^3, outside the safe box):
    # the walk must accept that node exactly when a_lim exceeds the node's bound
    mesh = I.uniform_mesh(8)
    rho = np.exp(0.5 * np.random.default_rng(9).standard_normal((1, 8, 8, 8)))
    B = oracle.tree_bmoments(mesh, rho)
    mom = oracle.tree_build(mesh, rho)
    ra = mom["n1_com"][0, 0]
    B2, B3 = B["n1"][0, 0]
    bmax = np.linalg.norm(np.full(3, 0.25) + np.abs(ra - 0.25))
    t = 7 * 64 + 7 * 8 + 7
    r = np.full(3, 7.5 / 8)
    d = np.linalg.norm(r - ra)
    bound = 1.0 / d ** 2 / (1 - bmax / d) ** 2 * (3 * B2 / d ** 2 - 2 * B3 / d ** 3)
    n_acc = oracle.gravity_walk(mesh, rho, np.array([t]), mac="mpe", a_lim=bound * (1 + 1e-9))[2]["interactions"]
    n_open = oracle.gravity_walk(mesh, rho, np.array([t]), mac="mpe", a_lim=bound * (1 - 1e-9))[2]["interactions"]
    assert n_open > n_acc
