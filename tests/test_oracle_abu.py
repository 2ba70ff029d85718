"""Pins for the oracle's Adaptive Block Update and block workload weights (Sec. 2.2.6)."""
import numpy as np

from paper_1708_06142_gb300 import inputs as I


def _case(seed=0):
    mesh = I.build_mesh(lambda lvl, lo, size: lvl < 2 or (lvl < 3 and lo[0] < 0.4))
    rng = np.random.default_rng(seed)
    return mesh, np.exp(0.5 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))


def test_corner_cells():
    from oracle import oracle as O
    c = O.abu_corner_cells(2)
    assert c.shape == (2, 8)
    assert set(c[0]) == {0, 7, 56, 63, 448, 455, 504, 511}
    np.testing.assert_array_equal(c[1] - c[0], 512)


def test_abu_limits(oracle):
    mesh, rho = _case()
    p_full, a_full, _ = oracle.gravity_walk(mesh, rho)
    # previous values from another density: a zero tolerance updates every block (= the full walk)
    rho_old = rho * np.exp(0.1 * np.random.default_rng(5).standard_normal(rho.shape))
    p_old, a_old, _ = oracle.gravity_walk(mesh, rho_old)
    p, a, upd, nint = oracle.abu_walk(mesh, rho, p_old, a_old, a_tol=0.0)
    assert upd.all()
    np.testing.assert_array_equal(p, p_full)
    np.testing.assert_array_equal(a, a_full)
    assert (nint > 0).all()
    # an infinite tolerance keeps every previous value
    p, a, upd, nint = oracle.abu_walk(mesh, rho, p_old, a_old, a_tol=np.inf)
    assert not upd.any() and (nint == 0).all()
    np.testing.assert_array_equal(a, a_old)
    # previous values of the same density: every corner matches exactly, nothing is updated
    p, a, upd, _ = oracle.abu_walk(mesh, rho, p_full, a_full, a_tol=1e-300)
    assert not upd.any()


def test_abu_updates_blocks_whose_corners_change(oracle):
    mesh, rho = _case(1)
    p_old, a_old, _ = oracle.gravity_walk(mesh, rho)
    amax = np.linalg.norm(a_old, axis=1).max()
    # add 10 % mass in one leaf-block: the corners of nearby blocks change most
    rho2 = rho.copy()
    rho2[3] *= 1.1
    p, a, upd, _ = oracle.abu_walk(mesh, rho2, p_old, a_old, a_tol=1e-2 * amax)
    assert upd[3] and 0 < upd.sum() < mesh.nleaf
    p_full, a_full, _ = oracle.gravity_walk(mesh, rho2)
    cells = (np.arange(mesh.nleaf * 512) // 512)
    np.testing.assert_array_equal(a[upd[cells]], a_full[upd[cells]])
    np.testing.assert_array_equal(a[~upd[cells]], a_old[~upd[cells]])
    # the kept blocks' error stays of the order of the tolerance at their corners
    c = oracle.abu_corner_cells(mesh.nleaf)[~upd]
    assert np.linalg.norm(a[c] - a_full[c], axis=-1).max() < 1e-2 * amax


def test_workload_weights():
    from oracle import oracle as O
    w = np.ones(3)
    n = np.array([0, 50, 100])
    for _ in range(400):
        w = O.workload_update(w, n)
    # fixed point: 2 + omega N / N_max, between 2 (no work) and 2 + omega (the busiest block)
    np.testing.assert_allclose(w, [2.0, 6.0, 10.0], rtol=1e-12)
    w1 = O.workload_update([4.0], [0], tau=10.0)
    np.testing.assert_allclose(w1, [4.0 * np.exp(-0.1) + 2.0 * (1 - np.exp(-0.1))], rtol=1e-15)
