"""Pins for the oracle's HEALPix RING pixelisation (Gorski et al. 2005, used in Sec. 2.3)."""
import numpy as np
import pytest


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_round_trip_and_ring_latitudes(oracle, nside):
    npix = 12 * nside * nside
    pix = np.arange(npix)
    z, phi = oracle.healpix_pix2ang(nside, pix)
    st = np.sqrt(1 - z * z)
    v = np.stack([st * np.cos(phi), st * np.sin(phi), z], 1)
    np.testing.assert_array_equal(oracle.healpix_vec2pix(nside, v), pix)
    rings = sorted(set(np.round(z, 12)), reverse=True)
    assert len(rings) == 4 * nside - 1
    expect = [1 - i * i / (3 * nside ** 2) for i in range(1, nside)] + \
             [4 / 3 - 2 * i / (3 * nside) for i in range(nside, 3 * nside + 1)] + \
             [-(1 - i * i / (3 * nside ** 2)) for i in range(nside - 1, 0, -1)]
    np.testing.assert_allclose(rings, expect, atol=1e-12)


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_equal_area(oracle, nside):
    rng = np.random.default_rng(nside)
    v = rng.standard_normal((600_000, 3))
    pix = oracle.healpix_vec2pix(nside, v)
    npix = 12 * nside * nside
    cnt = np.bincount(pix, minlength=npix)
    assert cnt.size == npix
    e = v.shape[0] / npix
    chi2 = ((cnt - e) ** 2 / e).sum()
    # chi^2 with npix-1 dof: mean npix-1, sd sqrt(2(npix-1)); a wrong boundary gives >> this
    assert chi2 < npix - 1 + 6 * np.sqrt(2 * (npix - 1))


def test_nside1_base_pixels(oracle):
    # nside = 1: pixels 0-3 north (z = 2/3), 4-7 equator (z = 0), 8-11 south (z = -2/3)
    z, phi = oracle.healpix_pix2ang(1, np.arange(12))
    np.testing.assert_allclose(z, [2 / 3] * 4 + [0] * 4 + [-2 / 3] * 4, atol=1e-14)
    np.testing.assert_allclose(phi[:4], np.pi / 4 * np.array([1, 3, 5, 7]))
    np.testing.assert_allclose(phi[4:8], np.pi / 2 * np.arange(4))
