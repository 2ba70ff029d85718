"""GPU parity for the Adaptive Block Update (Sec. 2.2.6): the FP64 walk against the oracle's ABU
composition (same kept blocks, same values), the FP32 walk within tolerance, the tolerance limits,
and the block workload weights against the oracle's recurrence."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _case(seed=1):
    mesh = I.build_mesh(lambda lvl, lo, size: lvl < 2 or (lvl < 3 and lo[0] < 0.4))
    rng = np.random.default_rng(seed)
    return mesh, np.exp(0.5 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))


def _solver(mesh, rho):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    return ts


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mac", ["bh", "ape"])
def test_abu_matches_oracle(oracle, precision, mac):
    import torch
    mesh, rho = _case()
    kw = dict(theta=0.5) if mac == "bh" else dict(a_lim=0.05)
    p_old, a_old, _ = oracle.gravity_walk(mesh, rho, mac=mac, **kw)
    amax = np.linalg.norm(a_old, axis=1).max()
    rho2 = rho.copy()
    rho2[3] *= 1.1
    p_ref, a_ref, upd, nint = oracle.abu_walk(mesh, rho2, p_old, a_old, a_tol=1e-2 * amax, mac=mac, **kw)
    assert 0 < upd.sum() < mesh.nleaf
    ts = _solver(mesh, rho2)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pot = torch.from_numpy(p_old).to(dt).cuda()
    acc = torch.from_numpy(a_old).to(dt).cuda().contiguous()
    n = ts.gravity_walk_abu(pot, acc, 1e-2 * amax, precision=precision, mac=mac, **kw)
    assert n == upd.sum()
    a = acc.double().cpu().numpy()
    p = pot.double().cpu().numpy()
    if precision == "fp64":
        np.testing.assert_allclose(a, a_ref, rtol=0, atol=1e-12 * amax)
        np.testing.assert_allclose(p, p_ref, rtol=1e-12, atol=1e-12 * np.abs(p_ref).max())
        w = ts.block_workload()
        np.testing.assert_allclose(w, oracle.workload_update(np.full(mesh.nleaf, 2.0), nint), rtol=1e-12)
    else:
        e = np.linalg.norm(a - a_ref, axis=1) / amax
        assert np.median(e) < 1e-6 and e.max() < 1e-4


def test_abu_tolerance_limits():
    import torch
    mesh, rho = _case(2)
    ts = _solver(mesh, rho)
    pot = torch.empty(mesh.ncell, dtype=torch.float64, device="cuda")
    acc = torch.empty(mesh.ncell, 3, dtype=torch.float64, device="cuda")
    ts.gravity_walk(pot, acc, precision="fp64")
    ts.sync()
    full_p, full_a = pot.clone(), acc.clone()
    # same density: the corners reproduce their previous values bit for bit, nothing is walked
    assert ts.gravity_walk_abu(pot, acc, 1e-300, precision="fp64") == 0
    assert torch.equal(acc, full_a)
    # zero tolerance with stale inputs: every block is walked, the result is the full walk
    acc.zero_()
    pot.zero_()
    assert ts.gravity_walk_abu(pot, acc, 0.0, precision="fp64") == mesh.nleaf
    assert torch.equal(acc, full_a) and torch.equal(pot, full_p)
    # infinite tolerance keeps everything
    acc.fill_(1.0)
    assert ts.gravity_walk_abu(pot, acc, float("inf"), precision="fp64") == 0
    assert bool((acc == 1.0).all())


def test_abu_argument_errors():
    import torch
    from paper_1708_06142_gb300.treesolver import TSError
    mesh, rho = _case()
    ts = _solver(mesh, rho)
    pot = torch.zeros(mesh.ncell, device="cuda")
    acc = torch.zeros(mesh.ncell, 3, device="cuda")
    with pytest.raises(TSError) as e:
        ts.gravity_walk_abu(pot, acc, -1.0)
    assert e.value.status == 1
    with pytest.raises(TSError) as e:
        ts.block_workload() if False else ts.gravity_walk_abu(pot, acc, float("nan"))
    assert e.value.status == 1
