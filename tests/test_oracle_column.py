"""Pins for the oracle's node-ray table and column-density walk (Sec. 2.3).

- every table entry's weights sum to one (the node's whole mass is distributed);
- a small node (psi -> 0) falls in the one pixel of its direction;
- the table is invariant under the symmetries shared by the cube and the HEALPix grid;
- the mean visual extinction (eq. av): equal columns N give A_V = k N; one blocked pixel out of
  N_PIX gives ln(N_PIX / (N_PIX - 1)) / 2.5; A_V lies between k min N and k mean N (Jensen) and
  grows with every column;
- the centre of a uniform sphere sees N_i = rho R in every pixel (discretisation error only);
- conservation: sum_i N_i Omega_pix = sum over cells m/d^2 + 4 pi rho dx/2 with every node opened;
- a uniform slab: polar pixels see rho H / |cos theta| averaged over the pixel.
"""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I


def test_table_weights_normalised_and_point_limit(oracle):
    w = oracle.noderay_table(2, ntheta=10, nphi=20, npsi=6, psi_min=1e-3, psi_max=1.0, nsub=8)
    np.testing.assert_allclose(w.sum(-1), 1.0, atol=1e-12)
    th = (np.arange(10) + 0.5) * np.pi / 10
    ph = (np.arange(20) + 0.5) * 2 * np.pi / 20
    T, P = np.meshgrid(th, ph, indexing="ij")
    v = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    pix = oracle.healpix_vec2pix(2, v).reshape(10, 20)
    small = w[:, :, 0, :]
    assert (np.take_along_axis(small, pix[..., None], -1)[..., 0] > 0.95).mean() > 0.9


def test_uniform_sphere_centre_column(oracle):
    mesh = I.uniform_mesh(32)
    c = np.array([16.5, 16.5, 16.5]) / 32
    x = mesh.cell_centres()
    r = np.sqrt(((x - c) ** 2).sum(-1))
    R = 0.3
    rho = np.where(r < R, 1.0, 0.0)
    t = np.array([int(np.argmin(r.reshape(-1)))])
    # exact sub-cube quadrature per node: only the staircase sphere's discretisation error is left
    cols, _ = oracle.column_walk(mesh, rho, t, nside=2, theta=0.0, table=None)
    assert np.abs(cols[0] / R - 1.0).max() < 0.06
    # the tabulated weights (nearest bin of 25 x 50 x 25) add ~10 % per pixel for nearby cells
    cols, _ = oracle.column_walk(mesh, rho, t, nside=2, theta=0.5)
    assert np.abs(cols[0] / R - 1.0).max() < 0.2
    assert abs(cols[0].mean() / R - 1.0) < 0.03


def test_column_conservation_all_cells(oracle):
    mesh = I.uniform_mesh(16)
    rng = np.random.default_rng(2)
    rho = np.exp(0.5 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))
    tg = I.sample_cells(mesh.ncell, 20, seed=3)
    cols, cnt = oracle.column_walk(mesh, rho, tg, nside=2, theta=0.0)
    assert cnt["interactions"] == tg.size * (mesh.ncell - 1)
    x = mesh.cell_centres().reshape(-1, 3)
    m = (rho * mesh.cell_volume()[:, None, None, None]).reshape(-1)
    omega = 4 * np.pi / 48
    for n, t in enumerate(tg):
        d2 = ((x - x[t]) ** 2).sum(1)
        d2[t] = np.inf
        expect = (m / d2).sum() + 4 * np.pi * rho.reshape(-1)[t] * 0.5 / 16
        assert cols[n].sum() * omega == pytest.approx(expect, rel=1e-12)


def test_uniform_slab_polar_pixels(oracle):
    # slab 0.375 < z < 0.625, x,y periodic (minimum image); the columns towards the poles are the
    # distances to the slab faces over |cos theta|, averaged over the pixel
    n = 32
    mesh = I.uniform_mesh(n, bc=(1, 1, 0))
    x = mesh.cell_centres()
    rho = np.where(np.abs(x[..., 2] - 0.5) < 0.125, 1.0, 0.0)
    xf = x.reshape(-1, 3)
    t = np.array([int(np.argmin(((xf - [0.515625, 0.515625, 0.484375]) ** 2).sum(1)))])
    zt = xf[t[0], 2]
    cols, _ = oracle.column_walk(mesh, rho, t, nside=2, theta=0.0, table=None, nsub=8)
    zc, _ = oracle.healpix_pix2ang(2, np.arange(48))
    for p in range(4):                       # north polar cap pixels, centres at z = 11/12
        assert cols[0, p] == pytest.approx((0.625 - zt) / abs(zc[p]), rel=0.03)
    for p in range(44, 48):                  # south polar cap
        assert cols[0, p] == pytest.approx((zt - 0.375) / abs(zc[p]), rel=0.03)


def test_table_symmetries(oracle):
    """The axis-aligned cube and the HEALPix grid share the symmetries z -> -z, y -> -y and the
    quarter turn about z; each maps table bins onto table bins and pixels onto pixels, so the
    weights must be equal under the matching pixel permutation (up to a quadrature sample that
    lies on a pixel boundary and falls on the other side after rounding: 1/nsub^3 each)."""
    nside, nt, nph, nps, nsub = 2, 8, 20, 4, 8
    w = oracle.noderay_table(nside, ntheta=nt, nphi=nph, npsi=nps, psi_min=1e-2, psi_max=1.0, nsub=nsub)
    npix = 12 * nside * nside
    z, ph = oracle.healpix_pix2ang(nside, np.arange(npix))
    s = np.sqrt(1 - z * z)
    v = np.stack([s * np.cos(ph), s * np.sin(ph), z], -1)
    tol = 2.5 / nsub ** 3

    def perm(f):   # pixel index of the image of every pixel centre
        return oracle.healpix_vec2pix(nside, f(v))

    # z -> -z: theta bin it -> nt - 1 - it
    pz = perm(lambda u: u * [1, 1, -1])
    assert np.abs(w[::-1][..., pz] - w).max() <= tol
    # y -> -y: phi bin ip -> nph - 1 - ip
    py = perm(lambda u: u * [1, -1, 1])
    assert np.abs(w[:, ::-1][..., py] - w).max() <= tol
    # quarter turn (x, y) -> (-y, x): phi bin ip -> ip + nph / 4
    pr = perm(lambda u: np.stack([-u[:, 1], u[:, 0], u[:, 2]], -1))
    rolled = np.roll(w, -(nph // 4), axis=1)       # rolled[:, ip] = w[:, ip + nph/4]
    assert np.abs(rolled[..., pr] - w).max() <= tol
    # and the permutations are not trivial (the test would pass vacuously otherwise)
    assert (pz != np.arange(npix)).any() and (pr != np.arange(npix)).any()


def test_column_av_closed_forms(oracle):
    k = 0.37
    for n in (0.0, 1e-3, 0.5, 7.0, 100.0):
        np.testing.assert_allclose(oracle.column_av(np.full((3, 48), n), k), k * n, rtol=1e-13, atol=1e-15)
    cols = np.zeros((1, 48))
    cols[0, 5] = 1e6                            # one pixel fully blocked
    np.testing.assert_allclose(oracle.column_av(cols), np.log(48 / 47) / 2.5, rtol=1e-13)
    rng = np.random.default_rng(3)
    cols = np.exp(rng.normal(0.0, 1.5, size=(200, 192)))
    av = oracle.column_av(cols, k)
    assert (av >= k * cols.min(-1) - 1e-12).all() and (av <= k * cols.mean(-1) + 1e-12).all()
    more = cols.copy()
    more[:, 7] *= 2.0
    grown = oracle.column_av(more, k)
    # strictly larger wherever pixel 7 still transmits a resolvable fraction of the light
    assert (grown >= av).all() and (grown > av)[2.5 * k * cols[:, 7] < 20].all()
