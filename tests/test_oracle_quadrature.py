"""Independent pins of the oracle's mixed-boundary Fourier integrals (Sec. 2.2.4): the closed forms
of the 2P1I integral (eqs. intij and int00, scaled as eq. intijscaled) and the Gauss-Legendre
quadrature of the 1P2I integrals (eq. int00p1 and its radial derivative) against adaptive quadrature
of the integrals as the paper defines them (eq. intdef and eq. int00p1), with scipy.  A wrong sign,
a dropped term, a transposed argument or too coarse a quadrature rule fails these at 1e-10.  Points
include the near field (R -> 0, z -> 0) and the edge of the Fourier cut-off."""
import numpy as np
import pytest

integrate = pytest.importorskip("scipy.integrate")
special = pytest.importorskip("scipy.special")

ZETA = np.pi ** 2 / 4.0          # zeta = pi^2 / (alpha Lx)^2 with alpha = 2 / Lx
U = np.sqrt(60.0 / ZETA)         # exp(-zeta U^2) = e^-60


def _quad(f):
    v, err = integrate.quad(f, 0.0, U, limit=2000, epsabs=1e-14, epsrel=1e-13)
    return v


@pytest.mark.parametrize("s", [0.0, 1.0, np.sqrt(2.0), 2.5, np.sqrt(10.0)])
@pytest.mark.parametrize("gam", [0.0, 1e-6, 0.3, 2.0, 7.0, 15.0])
def test_2p1i_fourier_integral_against_quadrature(oracle, s, gam):
    it, ip = oracle.fourier_2p1i(s, gam, ZETA)
    if s == 0.0:
        # eq. int00: the divergent constant dropped, I = -4 int e^{-zeta u^2} sin^2(gam u/2)/u^2
        want = -4.0 * _quad(lambda u: np.exp(-ZETA * u * u) * np.sinc(gam * u / (2 * np.pi)) ** 2 * (gam / 2) ** 2)
        dwant = -2.0 * _quad(lambda u: np.exp(-ZETA * u * u) * gam * np.sinc(gam * u / np.pi))
    else:
        sc = np.exp(-ZETA * s * s)
        want = sc * 2.0 * _quad(lambda u: np.exp(-ZETA * u * u) * np.cos(gam * u) / (s * s + u * u))
        dwant = sc * -2.0 * _quad(lambda u: np.exp(-ZETA * u * u) * u * np.sin(gam * u) / (s * s + u * u))
    assert abs(it - want) <= 1e-10 * max(1.0, abs(want)), (s, gam, it, want)
    assert abs(ip - dwant) <= 1e-10 * max(1.0, abs(dwant)), (s, gam, ip, dwant)


@pytest.mark.parametrize("l1", [0, 1, 2, 3])
@pytest.mark.parametrize("eta", [1e-6, 0.05, 0.7, 3.0, 12.0, 40.0])
def test_1p2i_integrals_against_quadrature(oracle, l1, eta):
    K, M = oracle.km_1p2i(l1, eta, ZETA)
    j0 = lambda q: special.j0(eta * q)
    j1 = lambda q: special.j1(eta * q)
    if l1 == 0:
        # regularised: int (J0(eta q) - 1) e^{-zeta q^2} / q dq (the divergent constant dropped)
        kw = _quad(lambda q: (j0(q) - 1.0) * np.exp(-ZETA * q * q) / q if q > 0 else 0.0)
    else:
        kw = _quad(lambda q: j0(q) * np.exp(-ZETA * q * q) * q / (l1 * l1 + q * q))
    mw = _quad(lambda q: j1(q) * np.exp(-ZETA * q * q) * q * q / (l1 * l1 + q * q))
    assert abs(K - kw) <= 1e-10 * max(1.0, abs(kw)), (l1, eta, K, kw)
    assert abs(M - mw) <= 1e-10 * max(1.0, abs(mw)), (l1, eta, M, mw)


def test_1p2i_l0_closed_form_far(oracle):
    # K(0, eta) = -(1/2) [gamma_E + ln(eta^2 / 4 zeta) + E1(eta^2 / 4 zeta)]: an exact identity
    for eta in (1e-3, 0.5, 4.0, 25.0):
        K, _ = oracle.km_1p2i(0, eta, ZETA)
        x = eta * eta / (4 * ZETA)
        want = -0.5 * (np.euler_gamma + np.log(x) + special.exp1(x))
        assert abs(K - want) <= 1e-10 * max(1.0, abs(want)), (eta, K, want)
