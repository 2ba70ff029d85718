"""Pins of the oracle's accuracy metrics (Sec. 3, eq. ea) against closed forms."""
import numpy as np
import pytest

from oracle import oracle as O


def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("n", [1, 3, 101, 1001])
def test_e_a_uniform_offsets(n):
    # |a_ref| = 2 everywhere, |a - a_ref| = 2 i / (n - 1): e_a takes the values i / (n - 1)
    rng = np.random.default_rng(n)
    ref = 2.0 * _unit(rng, n)
    d = np.arange(n) / max(n - 1, 1)
    acc = ref + 2.0 * d[rng.permutation(n), None] * _unit(rng, n)
    s = O.error_stats(acc=acc, acc_ref=ref)
    assert s["a_ref_max"] == pytest.approx(2.0, rel=1e-15)
    assert s["e_a_max"] == pytest.approx(d.max(), abs=1e-14)
    # order statistic at position q (n - 1) of i / (n - 1) is q itself
    assert s["e_a_median"] == pytest.approx(0.5 if n > 1 else 0.0, abs=1e-14)
    assert s["e_a_p99"] == pytest.approx(0.99 if n > 1 else 0.0, abs=1e-14)
    assert s["n_nonfinite"] == 0 and s["n"] == n


def test_normaliser_is_the_domain_maximum():
    # one large reference vector sets the scale of every cell's error (not the cell's own |a_ref|)
    ref = np.array([[1.0, 0, 0], [0, 10.0, 0], [0, 0, 0.1]])
    acc = ref + np.array([[0.5, 0, 0], [0, 0, 0], [0, 0, 0.05]])
    s = O.error_stats(acc=acc, acc_ref=ref)
    assert s["e_a_max"] == pytest.approx(0.05)
    assert s["e_a_median"] == pytest.approx(0.005)


def test_potential_modulo_constant():
    rng = np.random.default_rng(4)
    ref = -1.0 - rng.random(257)
    s = O.error_stats(pot=ref + 5.0, pot_ref=ref, mod_const=True)
    assert s["e_phi_max"] < 1e-14
    s = O.error_stats(pot=ref + 5.0, pot_ref=ref, mod_const=False)
    assert s["e_phi_median"] == pytest.approx(5.0 / np.abs(ref).max(), rel=1e-14)


def test_zero_reference_gives_absolute_error_and_nonfinite_count():
    acc = np.zeros((5, 3))
    acc[:, 0] = [0.0, 1.0, 2.0, 3.0, 4.0]
    s = O.error_stats(acc=acc, acc_ref=np.zeros((5, 3)))
    assert s["e_a_median"] == 2.0 and s["e_a_max"] == 4.0
    acc[2, 1] = np.nan
    s = O.error_stats(acc=acc, acc_ref=np.zeros((5, 3)))
    assert s["n_nonfinite"] == 1


def test_quantile_brute_force():
    # linear interpolation between the order statistics at floor/ceil of q (n - 1), written out
    rng = np.random.default_rng(7)
    for n in (2, 10, 999):
        ref = _unit(rng, n)
        acc = ref + 0.01 * rng.standard_normal((n, 3))
        s = O.error_stats(acc=acc, acc_ref=ref)
        e = sorted(np.linalg.norm(acc - ref, axis=1) / np.linalg.norm(ref, axis=1).max())
        for q, key in ((0.5, "e_a_median"), (0.99, "e_a_p99")):
            pos = q * (n - 1)
            lo = int(pos)
            hi = min(lo + 1, n - 1)
            assert s[key] == pytest.approx(e[lo] + (pos - lo) * (e[hi] - e[lo]), rel=1e-14)
