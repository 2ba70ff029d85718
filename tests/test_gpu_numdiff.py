"""Potential-only walks with the acceleration by numerical differentiation (Sec. 2.2.2) on the GPU:
the potential-only kernels give the full walk's potential bit for bit; the differentiation kernel
matches the oracle's stencil applied to the very same potential; end to end, against the FP64
oracle walk differentiated by the oracle."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I
from tests.gpu_util import e_a

pytestmark = pytest.mark.gpu


def _amr_mesh():
    def refine(lev, lo, sz):
        p = np.array([0.3, 0.6, 0.45])
        gap = np.linalg.norm(np.maximum(0.0, np.maximum(lo - p, p - (lo + sz))))
        return lev < 2 or (lev < 4 and gap < 0.12 / lev)
    return I.build_mesh(refine)


def _cases():
    rng = np.random.default_rng(3)
    out = []
    m, rho = I.sphere_32(seed=0, ncell_axis=16)
    out.append(("sphere16", m, rho))
    m = _amr_mesh()
    x, y, z = m.cell_centres().reshape(-1, 3).T
    rho = np.exp(-((x - 0.3) ** 2 + (y - 0.6) ** 2 + (z - 0.45) ** 2) / 0.02) + 1e-2
    out.append(("amr", m, rho.reshape(m.nleaf, 8, 8, 8) * np.exp(0.2 * rng.standard_normal((m.nleaf, 8, 8, 8)))))
    m = I.uniform_mesh(16, bc=(1, 1, 1))
    out.append(("periodic3p", m, np.exp(0.6 * rng.standard_normal((m.nleaf, 8, 8, 8)))))
    m = I.uniform_mesh(16, box=(1.0, 1.0, 2.0), bc=(1, 1, 0))
    out.append(("mixed2p1i", m, np.exp(0.6 * rng.standard_normal((m.nleaf, 8, 8, 8)))))
    return out


CASES = _cases()


def _walk(ts, mesh, precision, **kw):
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    pot = torch.empty(mesh.ncell, dtype=dt, device="cuda")
    acc = torch.empty(mesh.ncell, 3, dtype=dt, device="cuda")
    ts.gravity_walk(pot, acc, precision=precision, **kw)
    ts.sync()
    return pot.cpu().numpy().astype(np.float64), acc.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name,mesh,rho", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_potential_only_walk_and_differentiation(oracle, name, mesh, rho, precision):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(np.ascontiguousarray(rho).reshape(-1)).cuda())
    if any(mesh.bc):
        ts.ewald_field(32)
    macs = [dict(mac="bh", theta=0.5), dict(mac="ape", a_lim=1e-3)]
    if any(mesh.bc):
        macs.append(dict(mac="bh", theta=0.5, ewald="taylor"))
    for kw in macs:
        p_full, a_full = _walk(ts, mesh, precision, **kw)
        p_nd, a_nd = _walk(ts, mesh, precision, accel="numdiff", **kw)
        # the potential-only kernels form the same sums; the compiler may contract a product and a
        # sum into an FMA differently in the two kernels, so results agree to rounding of the sums
        # (periodic potentials cross zero: the tolerance is relative to the largest value)
        tol_p = 1e-13 if precision == "fp64" else 1e-6
        np.testing.assert_allclose(p_nd, p_full, rtol=0, atol=tol_p * np.abs(p_full).max())
        # the differentiation kernel against the oracle's stencil on the same potential values
        want = oracle.num_diff(mesh, p_nd)
        scale = np.abs(want).max()
        tol = 1e-12 if precision == "fp64" else 2e-6
        assert np.abs(a_nd - want).max() <= tol * scale, (name, kw, np.abs(a_nd - want).max() / scale)


@pytest.mark.parametrize("name,mesh,rho", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_numdiff_end_to_end_against_oracle(oracle, name, mesh, rho):
    """GPU potential-only walk + differentiation against the FP64 oracle walk's potential
    differentiated by the oracle (isolated BCs, BH theta = 0.5)."""
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    p_ref, a_direct, _ = oracle.gravity_walk(mesh, rho, mac="bh", theta=0.5)
    a_ref = oracle.num_diff(mesh, p_ref)
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(np.ascontiguousarray(rho).reshape(-1)).cuda())
    _, a64 = _walk(ts, mesh, "fp64", accel="numdiff")
    _, a32 = _walk(ts, mesh, "fp32", accel="numdiff")
    amax = np.linalg.norm(a_ref, axis=1).max()
    assert e_a(a64, a_ref, amax).max() < 1e-9
    e32 = e_a(a32, a_ref, amax)
    assert np.median(e32) <= 1e-3 and np.quantile(e32, 0.99) <= 1e-2, (np.median(e32), np.quantile(e32, 0.99))
    # for the record: the numerically differentiated field against the directly summed one
    ed = e_a(a_ref, a_direct)
    print(name, "numdiff vs direct: median e_a", np.median(ed), "max", ed.max())


def test_numdiff_rejected_where_unsupported():
    import torch
    from paper_1708_06142_gb300.treesolver import Batch, TreeSolver, TSError
    mesh, rho = I.sphere_32(seed=0, ncell_axis=16)
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    pot = torch.zeros(mesh.ncell, device="cuda")
    acc = torch.zeros(mesh.ncell, 3, device="cuda")
    with pytest.raises(TSError) as e:
        ts.gravity_walk_abu(pot, acc, 1e-3, accel="numdiff")
    assert e.value.status == 2
    p = ts.gravity_params(accel="numdiff")
    with pytest.raises(TSError) as e:
        Batch([ts]).run(gravity=p, pots=[pot], accs=[acc])
    assert e.value.status == 2
    p.accel = 7
    with pytest.raises(TSError) as e:
        ts.gravity_walk(pot, acc, params=p)
    assert e.value.status == 1
