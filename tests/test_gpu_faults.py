"""Failure detection on a GPU without provoking any GPU fault: allocation failures injected on the
host (TS_FAULT) at each allocation of an entry point, a damaged Ewald cache file that must be
regenerated, and a damaged surrogate file that must be rejected.  After every injected failure the
context stays usable and gives the same results as a clean run."""
import os

import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture
def fault():
    """Sets TS_FAULT for the duration of one call; always cleared afterwards."""
    def set_(v):
        if v is None:
            os.environ.pop("TS_FAULT", None)
        else:
            os.environ["TS_FAULT"] = v
    yield set_
    os.environ.pop("TS_FAULT", None)


def _walk(ts, n):
    import torch
    ts.ncell = n          # the binding learns ncell from a successful build only
    pot = torch.empty(n, device="cuda")
    acc = torch.empty(n, 3, device="cuda")
    ts.gravity_walk(pot, acc)
    ts.sync()
    return pot.cpu().numpy(), acc.cpu().numpy()


def test_tree_build_allocation_failures(fault):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver, TSError
    mesh, rho = I.sphere_32(ncell_axis=16)
    d = torch.from_numpy(rho.reshape(-1)).cuda()
    ref = TreeSolver(0)
    ref.tree_build(mesh, d)
    p_ref, a_ref = _walk(ref, mesh.ncell)
    ts = TreeSolver(0)
    # the mesh ingest allocates 12 device arrays: fail each one in turn, then all of them
    for k in list(range(1, 13)) + [None]:
        fault("tree_build" if k is None else f"tree_build:{k}")
        with pytest.raises(TSError) as e:
            ts.tree_build(mesh, d)
        assert e.value.status == 3, k
        fault(None)
        with pytest.raises(TSError) as e:    # no mesh survives a failed ingest
            _walk(ts, mesh.ncell)
        assert e.value.status == 5
    fault("tree_build:13")                    # beyond the last allocation: nothing fails
    ts.tree_build(mesh, d)
    fault(None)
    p, a = _walk(ts, mesh.ncell)
    np.testing.assert_array_equal(p, p_ref)
    np.testing.assert_array_equal(a, a_ref)


def test_ewald_and_taylor_allocation_failures(fault):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver, TSError
    mesh = I.uniform_mesh(16, bc=(1, 1, 1))
    rho = np.exp(0.5 * np.random.default_rng(3).standard_normal(mesh.ncell))
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho).cuda())
    for site in ("ewald_field:1", "ewald_field:2"):
        fault(site)
        with pytest.raises(TSError) as e:
            ts.ewald_field(16)
        assert e.value.status == 3
        fault(None)
        with pytest.raises(TSError) as e:     # the failed table is not left half-built
            _walk(ts, mesh.ncell)
        assert e.value.status == 5
    ts.ewald_field(16)
    pot = torch.empty(mesh.ncell, device="cuda")
    acc = torch.empty(mesh.ncell, 3, device="cuda")
    fault("taylor")
    with pytest.raises(TSError) as e:
        ts.gravity_walk(pot, acc, ewald="taylor")
    assert e.value.status == 3
    fault(None)
    ts.gravity_walk(pot, acc, ewald="taylor")
    ts.sync()
    assert np.isfinite(acc.cpu().numpy()).all()


def test_column_metrics_batch_and_surrogate_allocation_failures(fault):
    import torch
    from paper_1708_06142_gb300.treesolver import Batch, TreeSolver, TSError
    mesh, rho = I.sphere_32(ncell_axis=16)
    ts = TreeSolver(0)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    cols = torch.empty(mesh.ncell, 48, device="cuda")
    fault("noderay:2")
    with pytest.raises(TSError) as e:
        ts.column_walk(cols, ts.column_params(n_side=2))
    assert e.value.status == 3
    fault(None)
    ts.column_walk(cols, ts.column_params(n_side=2))
    ts.sync()
    assert np.isfinite(cols.cpu().numpy()).all()
    p, a = _walk(ts, mesh.ncell)
    pr = torch.from_numpy(p.astype(np.float64)).cuda()
    ar = torch.from_numpy(a.astype(np.float64)).cuda()
    fault("error_metrics")
    with pytest.raises(TSError) as e:
        ts.error_metrics(torch.from_numpy(p).cuda(), torch.from_numpy(a).cuda(), pr, ar)
    assert e.value.status == 3
    fault(None)
    st = ts.error_metrics(torch.from_numpy(p).cuda(), torch.from_numpy(a).cuda(), pr, ar)
    assert st["e_a_max"] == 0.0
    for k in (1, 5, 9):
        fault(f"batch_create:{k}")
        with pytest.raises(TSError) as e:
            Batch([ts])
        assert e.value.status == 3
    fault(None)
    Batch([ts])
    fault("surrogate:3")
    with pytest.raises(TSError) as e:
        ts.surrogate_train(n_samples=1 << 12, steps=2, batch=256)
    assert e.value.status == 3
    fault(None)
    ts.surrogate_train(n_samples=1 << 12, steps=2, batch=256)


def test_damaged_ewald_cache_is_regenerated(tmp_path):
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    mesh = I.uniform_mesh(16, box=(1.0, 1.0, 2.0), bc=(1, 1, 0))
    rho = torch.ones(mesh.ncell, dtype=torch.float64, device="cuda")
    path = str(tmp_path / "ewald.bin")
    ts = TreeSolver(0)
    ts.tree_build(mesh, rho)
    ts.ewald_field(12, cache_path=path)
    tab0, ext0 = ts.ewald_table()
    good = open(path, "rb").read()
    # a cache that loads gives the same table
    ts2 = TreeSolver(0)
    ts2.tree_build(mesh, rho)
    ts2.ewald_field(12, cache_path=path)
    np.testing.assert_array_equal(ts2.ewald_table()[0], tab0)
    # one flipped byte in the body: detected by the content hash, table regenerated, file rewritten
    bad = bytearray(good)
    bad[len(bad) // 2] ^= 0x40
    open(path, "wb").write(bytes(bad))
    ts3 = TreeSolver(0)
    ts3.tree_build(mesh, rho)
    ts3.ewald_field(12, cache_path=path)
    np.testing.assert_array_equal(ts3.ewald_table()[0], tab0)
    assert open(path, "rb").read() == good


def test_surrogate_file_round_trip_and_damage(tmp_path):
    import torch
    from oracle import mlp as omlp
    from paper_1708_06142_gb300.treesolver import TreeSolver, TSError
    ts = TreeSolver(0)
    p = omlp.init(seed=5).astype(np.float32)
    norm = np.array([1.5, 0.7, 0.9, 2.0, 0.1, -0.2, 0.05, 0.3], dtype=np.float32)
    ts.surrogate_set(p, norm, [0.5, 2.0])
    path = str(tmp_path / "net.bin")
    ts.surrogate_save(path)
    ts2 = TreeSolver(0)
    with pytest.raises(TSError) as e:         # nothing to save yet
        ts2.surrogate_save(str(tmp_path / "none.bin"))
    assert e.value.status == 5
    ts2.surrogate_load(path)
    p2, n2, b2 = ts2.surrogate_get()
    np.testing.assert_array_equal(p2, p)
    np.testing.assert_array_equal(n2, norm)
    np.testing.assert_array_equal(b2, [0.5, 2.0])
    x = torch.from_numpy(np.random.default_rng(0).uniform(-1, 1, (256, 4)).astype(np.float32)).cuda()
    o1, o2 = torch.empty(256, 4, device="cuda"), torch.empty(256, 4, device="cuda")
    ts.surrogate_eval(x, o1)
    ts2.surrogate_eval(x, o2)
    ts.sync(); ts2.sync()
    assert torch.equal(o1, o2)
    good = open(path, "rb").read()
    for where in (20, len(good) - 5):         # header field (b range) and a parameter byte
        bad = bytearray(good)
        bad[where] ^= 0x01
        open(path, "wb").write(bytes(bad))
        with pytest.raises(TSError) as e:
            ts2.surrogate_load(path)
        assert e.value.status == 1 and "hash" in str(e.value)
    open(path, "wb").write(good[:-4])         # truncated
    with pytest.raises(TSError) as e:
        ts2.surrogate_load(path)
    assert e.value.status == 1
    # the failed loads left the loaded network in place
    np.testing.assert_array_equal(ts2.surrogate_get()[0], p)
