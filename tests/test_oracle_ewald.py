"""Pins for the oracle's Ewald sums (Secs. 2.2.3-2.2.5, App. A).

- Madelung constant of a simple cubic lattice with a neutralising background:
  lim_{d->0} (phi - 1/|d|) = -2.837297479 / L (a textbook value, independent of alpha).
- alpha invariance of A = -grad phi for alpha Lx = 1, 2, 4 (a wrong term in either the real- or
  the Fourier-space sum breaks it); phi is alpha invariant for 3P (background term included).
- A = -grad phi by central differences of phi (checks the App. A forms against the potentials).
- far fields: an infinite sheet (2P1I) has |A_z| = 2 pi / (b Lx^2); a line mass (1P2I) has
  A_R = 2 / (Lx R) (Gauss's law); the series reaches them beyond 2 Lx.
- the 1P2I l1 = 0 integral with its divergent constant dropped has the closed form
  -1/2 [gamma_E + ln(eta^2/4 zeta) + E1(eta^2/4 zeta)] (checked through phi differences).
- symmetry: phi even, A odd, periodic along periodic axes.
"""
import numpy as np
import pytest

PTS = np.array([[0.13, 0.27, -0.31], [0.4, -0.1, 0.2], [0.05, 0.01, 0.02], [-0.22, 0.37, 0.44]])
CASES = [((1, 1, 1), (1.0, 1.0, 1.0)), ((1, 1, 1), (1.0, 1.5, 2.0)), ((1, 1, 0), (1.0, 1.0, 4.0)),
         ((1, 1, 0), (1.0, 2.0, 1.0)), ((1, 0, 0), (1.0, 1.0, 1.0))]


def test_madelung_constant(oracle):
    for L in (1.0, 2.0):
        phi, A = oracle.ewald((1, 1, 1), (L, L, L), [[0, 0, 0]], corr=True)
        assert phi[0] == pytest.approx(-2.837297479 / L, abs=1e-8)
        assert np.abs(A).max() < 1e-14


@pytest.mark.parametrize("bc,L", CASES)
def test_alpha_invariance(oracle, bc, L):
    res = [oracle.ewald(bc, L, PTS, alpha_lx=al, rcut2=40, kcut2=40) for al in (1.0, 2.0, 4.0)]
    for p, a in res[::2]:
        assert np.abs(a - res[1][1]).max() < 1e-9
        if bc == (1, 1, 1):
            assert np.abs(p - res[1][0]).max() < 1e-9
        else:  # regularised constant depends on alpha only
            dp = p - res[1][0]
            assert np.ptp(dp) < 1e-9


@pytest.mark.parametrize("bc,L", CASES)
def test_acceleration_is_minus_gradient(oracle, bc, L):
    h = 1e-5
    _, A = oracle.ewald(bc, L, PTS)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        pp, _ = oracle.ewald(bc, L, PTS + e)
        pm, _ = oracle.ewald(bc, L, PTS - e)
        np.testing.assert_allclose(-(pp - pm) / (2 * h), A[:, ax], rtol=1e-6, atol=1e-6)


def test_default_cutoffs_converged(oracle):
    for bc, L in CASES:
        p1, a1 = oracle.ewald(bc, L, PTS)
        p2, a2 = oracle.ewald(bc, L, PTS, rcut2=60, kcut2=40)
        assert np.abs(a1 - a2).max() < 1e-9 and np.abs(p1 - p2).max() < 1e-9


def test_symmetry_and_periodicity(oracle):
    # a shifted point lies outside the minimum-image cell, so the real-space image sum needs a
    # larger cut-off there than the paper's (which assumes minimum-image separations)
    for bc, L in CASES:
        p, a = oracle.ewald(bc, L, PTS, rcut2=60)
        pm, am = oracle.ewald(bc, L, -PTS, rcut2=60)
        np.testing.assert_allclose(pm, p, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(am, -a, rtol=1e-10, atol=1e-11)
        for ax in range(3):
            if bc[ax]:
                s = np.zeros(3)
                s[ax] = L[ax]
                ps, as_ = oracle.ewald(bc, L, PTS + s, rcut2=60)
                np.testing.assert_allclose(ps, p, atol=1e-10)
                np.testing.assert_allclose(as_, a, atol=1e-10)


def test_sheet_far_field_2p1i(oracle):
    # the far field is reached beyond 2 max(Lx, Ly): the slowest neglected Fourier mode decays as
    # exp(-2 pi |dz| / max(Lx, Ly))
    for b in (1.0, 2.0):
        L = (1.0, b, 8.0)
        d = np.array([[0.1, 0.2, 2.5 * b], [0.3, -0.2, -3.0 * b], [0.0, 0.0, 3.5 * b]])
        p, A = oracle.ewald((1, 1, 0), L, d)
        np.testing.assert_allclose(A[:, 2], np.sign(d[:, 2]) * 2 * np.pi / b, rtol=1e-5)
        assert np.abs(A[:, :2]).max() < 1e-5
        pf, Af = oracle.ewald_far((1, 1, 0), L, d)
        np.testing.assert_allclose(p, pf, atol=1e-5)
        # slope of phi between two far points is -2 pi / (b Lx^2) per unit |z|
        assert (p[2] - p[0]) / (d[2, 2] - d[0, 2]) == pytest.approx(-2 * np.pi / b, rel=1e-5)


def test_line_far_field_1p2i_gauss(oracle):
    d = np.array([[0.1, 2.2, 1.0], [0.3, -1.5, -2.5], [0.45, 0.0, 3.0]])
    p, A = oracle.ewald((1, 0, 0), (1.0, 1.0, 1.0), d)
    R = np.sqrt(d[:, 1] ** 2 + d[:, 2] ** 2)
    np.testing.assert_allclose(A[:, 1], 2 * d[:, 1] / R ** 2, rtol=1e-5, atol=1e-7)
    np.testing.assert_allclose(A[:, 2], 2 * d[:, 2] / R ** 2, rtol=1e-5, atol=1e-7)
    assert np.abs(A[:, 0]).max() < 1e-5


def test_1p2i_l0_term_closed_form(oracle):
    # phi(R1) - phi(R2) on the axis-perpendicular plane far from the real-space images equals
    # (2/Lx)[K0(eta1) - K0(eta2)] + (l1 != 0 terms, ~exp(-2 pi R / Lx) < 1e-5 at R > 2 Lx)
    sc = pytest.importorskip("scipy.special")
    zeta = np.pi ** 2 / 4

    def k0(eta):
        x = eta ** 2 / (4 * zeta)
        return -0.5 * (np.euler_gamma + np.log(x) + sc.exp1(x))

    R = np.array([2.1, 2.6, 3.2])
    d = np.stack([np.zeros(3), R, np.zeros(3)], 1)
    p, _ = oracle.ewald((1, 0, 0), (1.0, 1.0, 1.0), d)
    expect = 2.0 * k0(2 * np.pi * R)
    np.testing.assert_allclose(p - p[0], expect - expect[0], atol=1e-5)


def test_correction_is_phi_minus_point_mass(oracle):
    for bc, L in CASES:
        p, a = oracle.ewald(bc, L, PTS)
        c, ac = oracle.ewald(bc, L, PTS, corr=True)
        r = np.linalg.norm(PTS, axis=1)
        np.testing.assert_allclose(c, p - 1 / r, atol=1e-12)
        np.testing.assert_allclose(ac, a - PTS / r[:, None] ** 3, atol=1e-10)
        # near the origin the correction is smooth (no 1/r remnant)
        tiny = np.array([[1e-4, 0, 0], [0, 2e-4, -1e-4]])
        c0, a0 = oracle.ewald(bc, L, [[0, 0, 0]], corr=True)
        ct, at = oracle.ewald(bc, L, tiny, corr=True)
        assert np.abs(ct - c0).max() < 1e-6 and np.abs(at).max() < 1e-3


def test_table_interpolates_correction(oracle):
    tab, ext = oracle.ewald_table((1, 1, 0), (1.0, 1.0, 4.0), n=17)
    np.testing.assert_allclose(ext, [0.5, 0.5, 2.0])
    i, j, k = 3, 11, 6
    d = np.array([[ext[0] * i / 16, ext[1] * j / 16, ext[2] * k / 16]])
    c, ac = oracle.ewald((1, 1, 0), (1.0, 1.0, 4.0), d, corr=True)
    np.testing.assert_allclose(tab[i, j, k], [c[0], *ac[0]], rtol=1e-13, atol=1e-14)
