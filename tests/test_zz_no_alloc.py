"""The allocation-free zero-mean entry point (for callers that may not allocate device memory,
e.g. a host code whose allocator owns the device's memory budget).  Checked through the C ABI
against the zero_mean option of the gravity walk, on two calls in a row (the shared scratch array
keeps the previous call's contents, which must not leak into the next result).  This file is
collected last on purpose."""
import numpy as np
import pytest

from paper_1708_06142_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_zero_mean_noalloc_matches_walk_zero_mean_twice():
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver, TSError, zero_mean_noalloc
    # two uniform meshes, and an AMR mesh whose leaf-blocks (levels 3-5) have different cell
    # volumes, so that the volume weights change the mean
    amr, _ = I.plummer_amr(seed=1, max_level=5)
    meshes = [I.uniform_mesh(32, bc=(1, 1, 1)), I.uniform_mesh(16, box=(1.0, 1.0, 2.0), bc=(1, 1, 0)), amr]
    assert np.ptp(amr.cell_volume()) > 0
    rng = np.random.default_rng(4)
    for mesh in meshes:
        rho = np.exp(0.6 * rng.standard_normal((mesh.nleaf, 8, 8, 8)))
        ts = TreeSolver(0)
        ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
        if any(mesh.bc):
            ts.ewald_field(32)
        raw = torch.empty(mesh.ncell, device="cuda")
        ref = torch.empty(mesh.ncell, device="cuda")
        acc = torch.empty(mesh.ncell, 3, device="cuda")
        ts.gravity_walk(raw, acc, theta=0.5)
        ts.gravity_walk(ref, acc, theta=0.5, zero_mean=True)
        ts.sync()
        vol_np = np.repeat(mesh.cell_volume(), 512)
        vol = torch.from_numpy(vol_np).cuda()
        raw_np = raw.cpu().numpy().astype(np.float64)
        for call in range(2):
            pot = raw.clone()
            zero_mean_noalloc(pot, weights=vol if call == 0 else None)
            torch.cuda.synchronize()
            got = pot.cpu().numpy()
            if call == 0:   # volume weights: the walk's own zero-mean option
                want = ref.cpu().numpy()
                mean = float((vol_np * got).sum() / vol_np.sum())
            else:           # equal weights: the plain FP64 mean
                want = (raw_np - raw_np.mean()).astype(np.float32)
                mean = float(got.astype(np.float64).mean())
            # same tolerance as the batched-vs-single comparison: ~1 ulp of the O(1) potential
            np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-6 * max(np.abs(want).max(), 1.0))
            assert abs(mean) < 1e-6 * max(np.abs(want).max(), 1.0)
    with pytest.raises(TSError) as e:
        zero_mean_noalloc(torch.empty(16_777_217, device="cuda"))
    assert e.value.status == 1


def test_zero_mean_noalloc_random_weights_against_fp64_mean():
    """Non-uniform random weights over several scratch slices and a ragged tail, against the FP64
    weighted mean computed with numpy, on two calls in a row on torch's current stream."""
    import torch
    from paper_1708_06142_gb300.treesolver import zero_mean_noalloc
    rng = np.random.default_rng(9)
    n = 3 * 4096 + 123
    for call in range(2):
        p = (rng.standard_normal(n) + 5.0 * call).astype(np.float32)
        w = rng.uniform(0.0, 3.0, n) ** 3
        pot = torch.from_numpy(p).cuda()
        zero_mean_noalloc(pot, weights=torch.from_numpy(w).cuda())
        torch.cuda.synchronize()
        want = (p.astype(np.float64) - (w * p).sum() / w.sum()).astype(np.float32)
        np.testing.assert_allclose(pot.cpu().numpy(), want, rtol=1e-6, atol=1e-6)
