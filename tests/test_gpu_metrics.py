"""Device accuracy metrics (Sec. 3, eq. ea) through the C ABI against the oracle's numpy definition."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ["a_ref_max", "phi_ref_max", "e_a_median", "e_a_p99", "e_a_max", "e_phi_median", "e_phi_p99", "e_phi_max"]


def _ts():
    from paper_1708_06142_gb300.treesolver import TreeSolver
    return TreeSolver(0)


def _case(n, seed, dtype):
    rng = np.random.default_rng(seed)
    aref = rng.standard_normal((n, 3)) * rng.lognormal(size=(n, 1))
    pref = -1.0 - rng.random(n)
    acc = (aref + 1e-3 * rng.standard_normal((n, 3))).astype(dtype)
    pot = (pref + 1e-4 * rng.standard_normal(n) + 0.25).astype(dtype)
    return pot, acc, pref, aref


@pytest.mark.parametrize("n", [1, 2, 7, 1001, 65536 + 37, 1 << 21])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("mod_const", [False, True])
def test_metrics_match_oracle(oracle, n, dtype, mod_const):
    import torch
    pot, acc, pref, aref = _case(n, n + (dtype == np.float64), dtype)
    ts = _ts()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    e_out = torch.empty(2, n, dtype=torch.float64, device="cuda")
    got = ts.error_metrics(pot=T(pot), acc=T(acc), pot_ref=T(pref), acc_ref=T(aref), mod_const=mod_const, e_out=e_out)
    ref = oracle.error_stats(pot=pot, acc=acc, pot_ref=pref, acc_ref=aref, mod_const=mod_const)
    assert got["n"] == n and got["n_nonfinite"] == 0
    # the potential means are FP64 sums in different orders: |error| <= n eps max|phi| each, which
    # shifts every e_phi by up to 2 n eps max|phi| / max|phi_ref|
    phi_abs = 2 * n * np.finfo(np.float64).eps * max(np.abs(pot).max(), np.abs(pref).max()) / (ref["phi_ref_max"] or 1.0)
    for k in KEYS:
        tol = phi_abs if (mod_const and k.startswith("e_phi")) else 0.0
        assert got[k] == pytest.approx(ref[k], rel=1e-11, abs=max(tol, 1e-300)), k
    # per-entry errors, the same definition written out here for the FP64 inputs
    e = e_out.cpu().numpy()
    ea = np.linalg.norm(acc.astype(np.float64) - aref, axis=1) / ref["a_ref_max"]
    np.testing.assert_allclose(e[0], ea, rtol=1e-12, atol=0)


def test_metrics_single_pair_and_exact_order_statistics(oracle):
    import torch
    # e_a values i / (n - 1) exactly representable: median and p99 must be the exact order statistics
    n = 101
    aref = np.zeros((n, 3))
    aref[:, 0] = 1.0
    acc = aref.copy()
    acc[:, 1] = np.random.default_rng(3).permutation(np.arange(n) / 100.0 * 1.0)
    ts = _ts()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got = ts.error_metrics(acc=T(acc), acc_ref=T(aref))
    ref = oracle.error_stats(acc=acc, acc_ref=aref)
    assert got["e_a_median"] == ref["e_a_median"] == 0.5
    assert got["e_a_p99"] == ref["e_a_p99"]
    assert got["e_a_max"] == 1.0
    assert got["e_phi_median"] == 0.0 and got["phi_ref_max"] == 0.0


def test_metrics_zero_reference_and_nonfinite(oracle):
    import torch
    acc = np.zeros((5, 3))
    acc[:, 0] = [0.0, 1.0, 2.0, 3.0, 4.0]
    ts = _ts()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    got = ts.error_metrics(acc=T(acc), acc_ref=T(np.zeros((5, 3))))
    assert got["e_a_median"] == 2.0 and got["e_a_max"] == 4.0 and got["a_ref_max"] == 0.0
    acc[2, 1] = np.nan
    got = ts.error_metrics(acc=T(acc), acc_ref=T(np.zeros((5, 3))))
    assert got["n_nonfinite"] == 1


def test_metrics_argument_errors():
    import torch
    from paper_1708_06142_gb300.treesolver import TSError
    ts = _ts()
    a = torch.zeros(4, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ts.error_metrics()
    with pytest.raises(TSError) as e:
        ts.error_metrics(acc=a)                   # value without its reference
    assert e.value.status == 1
    with pytest.raises(ValueError):
        ts.error_metrics(acc=a, acc_ref=torch.zeros(5, 3, dtype=torch.float64, device="cuda"))
