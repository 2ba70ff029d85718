"""Pins of the oracle's numerical differentiation of the potential (Sec. 2.2.2, the alternative to
eq. accel): exactness of the second-order stencils on polynomials, the closed form of the central
difference of a sine wave on a periodic grid, and, on an AMR mesh, the guard rules (injection from
coarser cells, volume mean over finer cells) checked against a point-location brute force."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I


def test_quadratic_field_is_differentiated_exactly(oracle):
    # central and one-sided second-order differences are exact for quadratics, in the interior and
    # at the isolated edges, also on a cuboid box with cuboid cells
    for box in ((1.0, 1.0, 1.0), (1.0, 0.5, 2.0)):
        m = I.uniform_mesh(16, box=box)
        x, y, z = m.cell_centres().reshape(-1, 3).T
        pot = x ** 2 + 2 * y ** 2 - z ** 2 + 0.3 * x * y - 0.7 * y * z + 0.2 * x
        a = oracle.num_diff(m, pot)
        want = -np.stack([2 * x + 0.3 * y + 0.2, 4 * y + 0.3 * x - 0.7 * z, -2 * z - 0.7 * y], 1)
        np.testing.assert_allclose(a, want, atol=1e-12)


def test_sine_wave_on_periodic_grid(oracle):
    # a_x of phi = sin(k x) by central differences is -k cos(k x) sin(k dx)/(k dx), exactly
    m = I.uniform_mesh(32, bc=(1, 1, 1))
    x, y, z = m.cell_centres().reshape(-1, 3).T
    k = 2 * np.pi * 3
    dx = 1.0 / 32
    pot = np.sin(k * x) + 0.5 * np.cos(2 * np.pi * z)
    a = oracle.num_diff(m, pot)
    np.testing.assert_allclose(a[:, 0], -k * np.cos(k * x) * np.sin(k * dx) / (k * dx), atol=1e-12)
    np.testing.assert_allclose(a[:, 1], 0.0, atol=1e-12)
    kz = 2 * np.pi
    np.testing.assert_allclose(a[:, 2], 0.5 * kz * np.sin(kz * z) * np.sin(kz * dx) / (kz * dx), atol=1e-12)


def _containing_leaf(mesh, p):
    lf = mesh.leaves
    lo, sz = mesh.lo[lf], mesh.size[lf]
    inside = np.all((p >= lo) & (p < lo + sz), axis=1)
    return lf[np.nonzero(inside)[0][0]], np.nonzero(inside)[0][0]


def test_amr_guard_rules_against_point_location(oracle):
    """A linear potential on an AMR mesh with level jumps: wherever a guard cube is a same-level or
    finer region the stencil reproduces the gradient exactly (the volume mean of a linear field is
    its value at the cube's centre); where a coarser cell supplies the guard (injection), the value
    is that cell's centre value.  The expected stencil is rebuilt here by locating points."""
    def refine(lev, lo, sz):
        p = np.array([0.3, 0.6, 0.45])
        gap = np.linalg.norm(np.maximum(0.0, np.maximum(lo - p, p - (lo + sz))))   # point-to-block distance
        return lev < 2 or (lev < 4 and gap < 0.12 / lev)

    m = I.build_mesh(refine)
    assert len(set(m.level[m.leaves])) >= 3
    g = np.array([0.7, -1.3, 0.4])
    cen = m.cell_centres().reshape(-1, 3)
    pot = cen @ g + 2.0
    a = oracle.num_diff(m, pot)
    lf = m.leaves
    dx_leaf = m.size[lf] / 8
    cell_dx = np.repeat(dx_leaf, 512, axis=0)
    rng = np.random.default_rng(0)
    sample = rng.choice(m.ncell, 400, replace=False)
    n_inject = 0
    for c in sample:
        want = np.zeros(3)
        for ax in range(3):
            vals = {}
            for s in (-2, -1, 1, 2):
                p = cen[c].copy()
                p[ax] += s * cell_dx[c, ax]
                if p[ax] < 0 or p[ax] >= 1:
                    continue
                b, n = _containing_leaf(m, p)
                if np.all(dx_leaf[n] >= cell_dx[c] - 1e-15):
                    # the containing cell is as large or larger: its own centre value
                    q = np.floor((p - m.lo[b]) / dx_leaf[n])
                    vals[s] = (m.lo[b] + (q + 0.5) * dx_leaf[n]) @ g + 2.0
                    n_inject += bool(np.any(dx_leaf[n] > cell_dx[c] + 1e-15))
                else:
                    vals[s] = p @ g + 2.0       # mean of the linear field over the cube
            h = cell_dx[c, ax]
            if -1 in vals and 1 in vals:
                d = (vals[1] - vals[-1]) / (2 * h)
            elif 1 in vals:
                d = (-3 * pot[c] + 4 * vals[1] - vals[2]) / (2 * h)
            else:
                d = -(-3 * pot[c] + 4 * vals[-1] - vals[-2]) / (2 * h)
            want[ax] = -d
        np.testing.assert_allclose(a[c], want, atol=1e-10)
    assert n_inject > 0   # the sample includes coarser guards


def test_walk_potential_differentiated_approaches_direct_acceleration(oracle):
    # the tree potential differentiated numerically approaches the directly summed acceleration
    # inside a smooth density at second order in the cell size
    errs = []
    for n in (16, 32):
        m = I.uniform_mesh(n)
        x, y, z = m.cell_centres().reshape(-1, 3).T
        rho = np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) / 0.05).reshape(m.nleaf, 8, 8, 8)
        pot, acc = oracle.direct_sum(m, rho)
        a = oracle.num_diff(m, pot)
        inner = (np.abs(x - 0.5) < 0.2) & (np.abs(y - 0.5) < 0.2) & (np.abs(z - 0.5) < 0.2)
        errs.append(np.linalg.norm(a[inner] - acc[inner], axis=1).max() / np.linalg.norm(acc, axis=1).max())
    assert errs[1] < errs[0] / 2.5, errs
