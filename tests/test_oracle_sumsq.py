"""Pins of the oracle's SumSquare MAC walk (Sec. 2.2.1): the limits a_lim -> 0 (every node opened:
the N^2 sum) and a_lim -> infinity (only the nodes whose MPE bound does not apply are opened: the MPE
walk with an infinite limit), the rigorous bound |a - a_N2| <= sqrt(n) a_lim that the summed squares
imply (Cauchy-Schwarz over the n accepted nodes), more interactions for tighter limits, and the
queue limit."""
import numpy as np

from paper_1708_06142_gb300 import inputs as I


def _mesh():
    def refine(lev, lo, sz):
        return lev < 2 or (lev < 3 and lo[0] < 0.5)
    m = I.build_mesh(refine)
    rng = np.random.default_rng(11)
    rho = np.exp(0.8 * rng.standard_normal((m.nleaf, 8, 8, 8)))
    return m, rho


def test_sumsq_limits(oracle):
    m, rho = _mesh()
    tg = I.sample_cells(m.ncell, 80, seed=3)
    p0, a0, c0 = oracle.gravity_walk(m, rho, tg, mac="sumsq", a_lim=1e-300, queue_max=1 << 16)
    pd, ad = oracle.direct_sum(m, rho, tg)
    assert c0["interactions"] == tg.size * (m.ncell - 1) and c0["overflows"] == 0
    np.testing.assert_allclose(a0, ad, rtol=0, atol=1e-12 * np.abs(ad).max())
    np.testing.assert_allclose(p0, pd, rtol=1e-12)
    # an infinite limit opens only the nodes whose bound does not apply: the MPE walk with a_lim = inf
    pi, ai, ci = oracle.gravity_walk(m, rho, tg, mac="sumsq", a_lim=1e300)
    pm, am, cm = oracle.gravity_walk(m, rho, tg, mac="mpe", a_lim=1e300)
    assert ci["interactions"] == cm["interactions"]
    np.testing.assert_allclose(ai, am, rtol=0, atol=1e-13 * np.abs(am).max())


def test_sumsq_error_bound_and_monotone(oracle):
    m, rho = _mesh()
    tg = I.sample_cells(m.ncell, 120, seed=4)
    _, ad = oracle.direct_sum(m, rho, tg)
    amax = np.linalg.norm(ad, axis=1).max()
    prev = None
    for eps in (1e-1, 1e-2, 1e-3):
        a_lim = eps * amax
        _, a, c = oracle.gravity_walk(m, rho, tg, mac="sumsq", a_lim=a_lim)
        err = np.linalg.norm(a - ad, axis=1)
        # per target, sum_i Delta_i^2 <= a_lim^2 over its n_i <= n accepted nodes, so the error
        # (at most sum_i Delta_i) is at most sqrt(n_i) a_lim; the mean count bounds sqrt(n_i) loosely
        n_per = c["interactions"] / tg.size
        assert np.all(err <= np.sqrt(n_per * 4) * a_lim), (eps, err.max() / a_lim)
        if prev is not None:
            assert c["interactions"] > prev[0] and np.median(err) < prev[1]
        prev = (c["interactions"], np.median(err))


def test_sumsq_queue_limit(oracle):
    m, rho = _mesh()
    tg = I.sample_cells(m.ncell, 20, seed=5)
    _, a, c = oracle.gravity_walk(m, rho, tg, mac="sumsq", a_lim=1e-12, queue_max=24)
    assert c["overflows"] > 0 and np.isfinite(a).all()
    _, _, c2 = oracle.gravity_walk(m, rho, tg, mac="sumsq", a_lim=1e-12, queue_max=1 << 16)
    assert c2["overflows"] == 0 and c2["interactions"] > c["interactions"]
