"""Checks against values the paper prints (tests/golden/paper_values.json, each entry citing its
passage): defaults of the walk, the far-field accuracy claim of Sec. 2.2.5 for the oracle's Ewald
series, the HEALPix pixel count, and the workload-weight parameters."""
import json
import os

import numpy as np
import pytest

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_walk_defaults_are_the_papers():
    import ctypes as C
    from paper_1708_06142_gb300 import treesolver as T
    T.load()
    p = T.TSGravityParams()
    T._lib.ts_gravity_params_default(C.byref(p))
    assert p.theta == GOLDEN["bh_theta_default"]["value"]
    assert p.safe_box == GOLDEN["safe_box_default"]["value"]


@pytest.mark.parametrize("b", [0.5, 1.0])
def test_far_field_claim_2p1i(oracle, b):
    # at |dz| beyond 2 Lx the analytic sheet form and the series agree to 1e-4 in acceleration
    g = GOLDEN["far_field_2p1i"]
    L = (1.0, b, 8.0)
    rng = np.random.default_rng(1)
    z = g["distance_in_Lx"] * (1.0 + rng.uniform(0.0, 1.0, 64))
    d = np.stack([rng.uniform(-0.5, 0.5, 64), rng.uniform(-0.5 * b, 0.5 * b, 64), z * rng.choice([-1, 1], 64)], 1)
    _, A = oracle.ewald((1, 1, 0), L, d)
    _, Af = oracle.ewald_far((1, 1, 0), L, d)
    err = np.linalg.norm(A - Af, axis=1) / np.linalg.norm(A, axis=1)
    assert err.max() < g["max_rel_acc_err"], err.max()


def test_far_field_claim_1p2i(oracle):
    g = GOLDEN["far_field_1p2i"]
    rng = np.random.default_rng(2)
    R = g["distance_in_Lx"] * (1.0 + rng.uniform(0.0, 1.0, 64))
    ang = rng.uniform(0, 2 * np.pi, 64)
    d = np.stack([rng.uniform(-0.5, 0.5, 64), R * np.cos(ang), R * np.sin(ang)], 1)
    _, A = oracle.ewald((1, 0, 0), (1.0, 8.0, 8.0), d)
    _, Af = oracle.ewald_far((1, 0, 0), (1.0, 8.0, 8.0), d)
    err = np.linalg.norm(A - Af, axis=1) / np.linalg.norm(A, axis=1)
    assert err.max() < g["max_rel_acc_err"], err.max()


def test_npix_of_nside(oracle):
    g = GOLDEN["npix_of_nside"]
    for tr, npix in zip(g["tr_nSide"], g["N_PIX"]):
        nside = 2 ** (tr - 1)          # the library's n_side = 2^(tr_nSide - 1)
        pix = oracle.healpix_vec2pix(nside, np.random.default_rng(tr).standard_normal((20000, 3)))
        assert pix.max() + 1 == npix and len(np.unique(pix)) == npix


def test_workload_parameters(oracle):
    g = GOLDEN["abu_workload"]
    # a block with no work relaxes to w_min, the busiest to w_min + omega, at rate exp(-1/tau)
    w = oracle.workload_update([g["w_min"] + g["omega_wl"], g["w_min"]], [0, 1])
    f = np.exp(-1.0 / g["tau_wl"])
    np.testing.assert_allclose(w, [(g["w_min"] + g["omega_wl"]) * f + (1 - f) * g["w_min"],
                                   g["w_min"] * f + (1 - f) * (g["w_min"] + g["omega_wl"])], rtol=1e-15)
