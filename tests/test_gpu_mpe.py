"""GPU parity for the MPE MAC (Sec. 2.2.1, eq. mpe with p = 1): the FP64 walk against the FP64
oracle walk with the same MAC (same accepted nodes, so the same interaction count), the FP32 walk
against it within the accuracy target, periodic BCs, and argument errors."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I
from tests.gpu_util import e_a, run_gravity

pytestmark = pytest.mark.gpu


def _amr(seed=0):
    mesh = I.build_mesh(lambda lvl, lo, size: lvl < 2 or (lvl < 4 and np.linalg.norm(lo + size / 2 - 0.3) < 0.3))
    rng = np.random.default_rng(seed)
    return mesh, np.exp(0.8 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))


@pytest.mark.parametrize("frac", [1e-2, 1e-3])
def test_fp64_mpe_walk_matches_oracle(oracle, frac):
    mesh, rho = _amr()
    _, a_ref0, _ = oracle.gravity_walk(mesh, rho, theta=0.5)
    amax = np.linalg.norm(a_ref0, axis=1).max()
    p_ref, a_ref, cnt = oracle.gravity_walk(mesh, rho, mac="mpe", a_lim=frac * amax)
    _, p64, a64, st = run_gravity(mesh, rho, precision="fp64", mac="mpe", a_lim=frac * amax)
    assert st["interactions"] == cnt["interactions"]
    assert st["mac_tests"] == cnt["mac_tests"]
    assert e_a(a64, a_ref).max() < 1e-11
    np.testing.assert_allclose(p64, p_ref, rtol=1e-11, atol=1e-12 * np.abs(p_ref).max())


def test_fp32_mpe_walk_against_oracle(oracle):
    mesh, rho = _amr(1)
    _, a0, _ = oracle.gravity_walk(mesh, rho, theta=0.5)
    a_lim = 1e-3 * np.linalg.norm(a0, axis=1).max()
    _, a_ref, cnt = oracle.gravity_walk(mesh, rho, mac="mpe", a_lim=a_lim)
    _, _, a32, st = run_gravity(mesh, rho, precision="fp32", mac="mpe", a_lim=a_lim)
    e = e_a(a32, a_ref)
    assert np.median(e) < 1e-6 and np.quantile(e, 0.99) < 1e-4, (np.median(e), e.max())
    assert abs(st["interactions"] - cnt["interactions"]) <= 1e-4 * cnt["interactions"]


def test_mpe_walk_meets_accuracy_target(oracle):
    # against the N^2 sum on sampled cells, at a limit of 1e-4 of the largest acceleration
    mesh, rho = _amr(2)
    tg = I.sample_cells(mesh.ncell, 256, seed=3)
    _, a_dir = oracle.direct_sum(mesh, rho, tg)
    amax = np.linalg.norm(a_dir, axis=1).max()
    _, _, a_mpe, st = run_gravity(mesh, rho, precision="fp32", mac="mpe", a_lim=1e-4 * amax)
    e = np.linalg.norm(a_mpe[tg] - a_dir, axis=1) / amax
    assert np.median(e) < 1e-3


def test_mpe_periodic_table(oracle):
    mesh = I.uniform_mesh(16, bc=(1, 1, 1))
    rho = np.exp(0.7 * np.random.default_rng(4).standard_normal((mesh.nleaf, 8, 8, 8)))
    tab = oracle.ewald_table((1, 1, 1), (1.0, 1.0, 1.0), n=64)
    _, a0, _ = oracle.gravity_walk(mesh, rho, ewald="table", table=tab)
    a_lim = 1e-3 * np.linalg.norm(a0, axis=1).max()
    _, a_ref, cnt = oracle.gravity_walk(mesh, rho, mac="mpe", a_lim=a_lim, ewald="table", table=tab)
    _, _, a64, st = run_gravity(mesh, rho, precision="fp64", ewald_n=64, mac="mpe", a_lim=a_lim)
    assert st["interactions"] == cnt["interactions"]
    assert e_a(a64, a_ref).max() < 1e-9


def test_mpe_argument_errors():
    import torch
    from paper_1708_06142_gb300.treesolver import TSError, TreeSolver
    mesh, rho = _amr()
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    pot = torch.empty(mesh.ncell, device="cuda")
    acc = torch.empty(mesh.ncell, 3, device="cuda")
    with pytest.raises(TSError) as e:
        ts.gravity_walk(pot, acc, mac="mpe", a_lim=0.0)
    assert e.value.status == 1
