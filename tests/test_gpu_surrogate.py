"""GPU tests of the learned Ewald correction (2P1I): forward pass and gradients of the BF16
tensor-core kernels against the FP64 oracle network, training against the FP64 Ewald series (three
training seeds), the learned-correction walk against the series walk, and what one network for the
whole aspect range buys against the per-aspect 64^3 table."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1708_06142_gb300 import inputs as I
from tests.gpu_util import e_a, run_gravity

pytestmark = pytest.mark.gpu


def _solver():
    from paper_1708_06142_gb300.treesolver import TreeSolver
    return TreeSolver(0)


def test_forward_matches_fp64_oracle():
    import torch
    ts = _solver()
    rng = np.random.default_rng(0)
    p = omlp.init(seed=3).astype(np.float32)
    norm = np.array([1.5, 0.7, 0.9, 2.0, 0.1, -0.2, 0.05, 0.3], dtype=np.float32)
    ts.surrogate_set(p, norm, [0.5, 2.0])
    x = rng.uniform(-1, 1, (1000, 4)).astype(np.float32)
    out = torch.empty(1000, 4, device="cuda")
    ts.surrogate_eval(torch.from_numpy(x).cuda(), out)
    ts.sync()
    # oracle with the same BF16-rounded inputs and weights (the kernels' operand precision)
    bfr = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float32)).bfloat16().float().numpy().astype(np.float64)
    layers = omlp.unpack(p.astype(np.float64))
    pq = omlp.pack([(bfr(W), b) for W, b in layers])
    ref = omlp.forward(pq, bfr(x)) * norm[:4] + norm[4:]
    got = out.cpu().numpy()
    err = np.abs(got - ref) / (np.abs(ref).max(0) + 1e-12)
    assert np.median(err) < 3e-3 and err.max() < 3e-2, (np.median(err), err.max())


def test_gradients_match_fp64_oracle():
    import torch
    ts = _solver()
    rng = np.random.default_rng(1)
    p = omlp.init(seed=4).astype(np.float32)
    ts.surrogate_set(p, np.array([1, 1, 1, 1, 0, 0, 0, 0], dtype=np.float32), [0.5, 2.0])
    n = 512
    x = rng.uniform(-1, 1, (n, 4)).astype(np.float32)
    t = rng.standard_normal((n, 4)).astype(np.float32)
    loss, g = ts.surrogate_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    lref, gref = omlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(lref, rel=2e-2)
    cos = float(g @ gref / (np.linalg.norm(g) * np.linalg.norm(gref)))
    rel = float(np.linalg.norm(g - gref) / np.linalg.norm(gref))
    assert cos > 0.999 and rel < 3e-2, (cos, rel)


@pytest.fixture(scope="module", params=[7, 8, 9], ids=["seed7", "seed8", "seed9"])
def trained(request):
    # three training seeds: the accuracy must not depend on a lucky one
    ts = _solver()
    loss = ts.surrogate_train(b_min=0.5, b_max=2.0, n_samples=1 << 20, steps=1000000, batch=4096, lr=3e-3,
                              seed=request.param, z_power=2.0)
    p, norm, br = ts.surrogate_get()
    return ts, loss, p, norm, br


def _series_points(oracle, b, n, seed):
    rng = np.random.default_rng(seed)
    F = 2 * max(1.0, b)
    d = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.5 * b, 0.5 * b, n), rng.uniform(-F, F, n)], 1)
    c, ac = oracle.ewald((1, 1, 0), (1.0, b, 8.0), d, corr=True)
    return d, np.concatenate([c[:, None], ac], 1)


def test_trained_network_against_series(oracle, trained):
    import torch
    ts, loss, p, norm, br = trained
    assert loss < 1e-4
    for b in (0.6, 1.0, 1.7):
        d, ref = _series_points(oracle, b, 2000, seed=int(10 * b))
        f = omlp.features(d, 1.0, b, br[0], br[1]).astype(np.float32)
        out = torch.empty(len(d), 4, device="cuda")
        ts.surrogate_eval(torch.from_numpy(f).cuda(), out)
        ts.sync()
        got = out.cpu().numpy()
        got[:, 1:] *= np.sign(d)          # odd components: restore the sign of the folded value
        err = np.abs(got - ref) / np.abs(ref).max(0)
        assert np.median(err) < 5e-3, (b, np.median(err, 0))
        # the FP64 oracle network with the exported weights agrees with the device network
        ref_net = omlp.forward(p.astype(np.float64), f.astype(np.float64)) * norm[:4] + norm[4:]
        ref_net[:, 1:] *= np.sign(d)
        assert np.median(np.abs(ref_net - got) / np.abs(ref).max(0)) < 5e-3


def test_one_network_for_the_aspect_range_against_64_tables(oracle, trained):
    """What the network buys, measured against the 64^3 correction table the walk actually uses:
    one network of 8,900 parameters (17.8 KB in BF16) serves every box aspect b in [0.5, 2], where a
    table (64^3 float4 = 4 MB on the device plus its FP64 master) is built per aspect.  The table is
    the faster lookup (and on the 256^3 disk the more accurate, see test_gpu_full_size); the network
    meets the accuracy target at every aspect with 1/235 of one table's memory.  Both walks' errors
    and times are printed."""
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    ts0, loss, p, norm, br = trained
    assert 8900 * 2 * 235 < 64 ** 3 * 16
    for b in (0.6, 1.0, 1.7):
        mesh = I.uniform_mesh(16, box=(1.0, b, 4.0), bc=(1, 1, 0))
        rng = np.random.default_rng(int(10 * b))
        z = mesh.cell_centres()[..., 2]
        rho = np.exp(-np.abs(z - 2) / 0.2) * np.exp(0.3 * rng.standard_normal(z.shape))
        tg = I.sample_cells(mesh.ncell, 200, seed=7)
        _, a_ref, _ = oracle.gravity_walk(mesh, rho, tg, ewald="series")
        ts = TreeSolver(0)
        ts.surrogate_set(p, norm, br)
        ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
        pot = torch.empty(mesh.ncell, device="cuda")
        acc = torch.empty(mesh.ncell, 3, device="cuda")
        ts.gravity_walk(pot, acc, ewald="mlp")
        ts.sync()
        t_net = ts.stats()["walk_ms"]
        e = e_a(acc.cpu().numpy().astype(np.float64)[tg], a_ref)
        tst, _, a_t, st = run_gravity(mesh, rho, precision="fp32", ewald_n=64)
        e_t = e_a(a_t[tg], a_ref)
        print(f"b={b}: network median e_a {np.median(e):.3g} ({t_net:.2f} ms), "
              f"64^3 table {np.median(e_t):.3g} ({st['walk_ms']:.2f} ms)")
        assert np.median(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2, (b, np.median(e), np.quantile(e, 0.99))
        assert np.median(e_t) <= 1e-3


def test_walk_with_learned_correction(oracle, trained):
    ts0, loss, p, norm, br = trained
    mesh = I.uniform_mesh(16, box=(1.0, 1.0, 4.0), bc=(1, 1, 0))
    rng = np.random.default_rng(5)
    z = mesh.cell_centres()[..., 2]
    rho = np.exp(-np.abs(z - 2) / 0.3) * np.exp(0.3 * rng.standard_normal(z.shape))
    tg = I.sample_cells(mesh.ncell, 300, seed=6)
    p_ref, a_ref, _ = oracle.gravity_walk(mesh, rho, tg, ewald="series")
    import torch
    from paper_1708_06142_gb300.treesolver import TreeSolver
    ts = TreeSolver(0)
    ts.surrogate_set(p, norm, br)
    ts.tree_build(mesh, torch.from_numpy(rho.reshape(-1)).cuda())
    pot = torch.empty(mesh.ncell, device="cuda")
    acc = torch.empty(mesh.ncell, 3, device="cuda")
    ts.gravity_walk(pot, acc, ewald="mlp")
    ts.sync()
    a = acc.cpu().numpy().astype(np.float64)[tg]
    e = e_a(a, a_ref)
    # The network's fit (RMS ~0.02-0.1 % of max |A| on the separations of the test points) leaves
    # the walk well inside the target (median e_a <= 1e-3) for each training seed; the table walk
    # stays below 1e-4.
    assert np.median(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2, (np.median(e), np.quantile(e, 0.99))
    # the table walk on the same mesh, for the record
    _, p_t, a_t, _ = run_gravity(mesh, rho, precision="fp32", ewald_n=64)
    print("median e_a: network", np.median(e), "table", np.median(e_a(a_t[tg], a_ref)))


def test_training_is_deterministic():
    # the CTAs' partial gradients are summed in a fixed order: the same seed gives the same network
    nets = []
    for _ in range(2):
        ts = _solver()
        ts.surrogate_train(b_min=0.5, b_max=2.0, n_samples=1 << 16, steps=2000, batch=4096, lr=3e-3, seed=11)
        nets.append(ts.surrogate_get()[0])
    np.testing.assert_array_equal(nets[0], nets[1])
