"""Pins for the oracle's first-order Taylor table of the Ewald correction (Sec. 2.2.5, approach 2).

- Laplacian: the correction C = phi - 1/|d| satisfies lap C = 4 pi / V for 3P (the neutralising
  background; the point masses of the lattice cancel against 1/|d| at the origin and lie outside
  the folded domain elsewhere) and lap C = 0 for 2P1I and 1P2I (no background; the sheet and line
  modes are part of the lattice sum).  J = dA_c/dd = -Hessian(C), so trace J = -4 pi / V or 0.
- J against central differences of the tabulated A_c between neighbouring grid points (second
  order in the grid spacing): catches a misplaced off-diagonal entry, which the trace cannot.
- the grid values equal the trilinear table's (same series at the same points).
- a walk with the Taylor lookup converges to the series walk at second order in the spacing.
"""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

CASES = [((1, 1, 1), (1.0, 1.0, 1.0)), ((1, 1, 1), (1.0, 1.5, 2.0)), ((1, 1, 0), (1.0, 1.0, 4.0)),
         ((1, 1, 0), (1.0, 2.0, 1.0)), ((1, 0, 0), (1.0, 1.0, 1.0))]


@pytest.mark.parametrize("bc,L", CASES)
def test_trace_is_minus_laplacian(oracle, bc, L):
    tab, ext = oracle.ewald_taylor_table(bc, L, n=9)
    tr = tab[..., 4] + tab[..., 7] + tab[..., 9]
    want = -4 * np.pi / np.prod(L) if bc == (1, 1, 1) else 0.0
    scale = np.abs(tab[..., 4:]).max()
    assert np.abs(tr - want).max() < 1e-6 * scale


@pytest.mark.parametrize("bc,L", CASES)
def test_jacobian_matches_table_differences(oracle, bc, L):
    n = 33
    tab, ext = oracle.ewald_taylor_table(bc, L, n=n)
    h = ext / (n - 1)
    A = tab[..., 1:4]
    J = tab[..., 4:]
    full = np.stack([np.stack([J[..., 0], J[..., 1], J[..., 2]], -1),
                     np.stack([J[..., 1], J[..., 3], J[..., 4]], -1),
                     np.stack([J[..., 2], J[..., 4], J[..., 5]], -1)], -2)   # [..., i, j] = dA_i/dd_j
    sl = (slice(1, -1),) * 3
    scale = np.abs(full).max()
    for j in range(3):
        fwd = [slice(1, -1)] * 3
        bwd = [slice(1, -1)] * 3
        fwd[j] = slice(2, None)
        bwd[j] = slice(0, -2)
        diff = (A[tuple(fwd)] - A[tuple(bwd)]) / (2 * h[j])          # dA_i/dd_j for every i
        err = np.abs(diff - full[sl][..., :, j]).max()
        assert err < 2e-2 * scale, (j, err, scale)


def test_grid_values_equal_trilinear_table(oracle):
    tt, e1 = oracle.ewald_taylor_table((1, 1, 0), (1.0, 1.0, 4.0), n=9)
    t4, e2 = oracle.ewald_table((1, 1, 0), (1.0, 1.0, 4.0), n=9)
    np.testing.assert_array_equal(e1, e2)
    np.testing.assert_array_equal(tt[..., :4], t4)


def test_taylor_walk_converges_at_second_order(oracle):
    mesh, rho = I.sphere_32(seed=0, ncell_axis=16)
    mesh = I.Mesh(mesh.level, mesh.child, mesh.lo, mesh.size, bc=(1, 1, 1))
    tg = I.sample_cells(mesh.ncell, 48, seed=3)
    p_ser, a_ser, _ = oracle.gravity_walk(mesh, rho, tg, ewald="series")
    amax = np.linalg.norm(a_ser, axis=1).max()
    errs, perrs = [], []
    # n - 1 odd keeps the cell separations (multiples of 1/16) off the grid points (multiples of
    # 1/(2 (n - 1))); spacing ratios 17/9 and 35/17
    for n in (10, 18, 36):
        tab = oracle.ewald_taylor_table((1, 1, 1), (1.0, 1.0, 1.0), n=n)
        p, a, _ = oracle.gravity_walk(mesh, rho, tg, ewald="taylor", table=tab)
        errs.append(np.sqrt(np.mean(np.sum((a - a_ser) ** 2, axis=1))) / amax)
        perrs.append(np.sqrt(np.mean((p - p_ser) ** 2)) / np.abs(p_ser).max())
    # second-order remainder: error ratios near (17/9)^2 = 3.6 and (35/17)^2 = 4.2
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5, errs
    assert errs[2] < 1e-4, errs
    assert perrs[0] / perrs[1] > 2.5 and perrs[1] / perrs[2] > 2.5, perrs
