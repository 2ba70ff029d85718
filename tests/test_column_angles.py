"""Host checks of the column walk's direction angles (Sec. 2.3 table lookup, bins in theta and phi).

The kernel takes theta = acos u_z and phi = atan2(y, x) from the polynomials `col_acos` and
`col_phi` of `csrc/ts_column_dev.cuh` instead of acosf / atan2f.  These tests read their coefficients
from that source, evaluate the same FMA chains in FP32 with numpy (each fused multiply-add formed
exactly in FP64 and rounded once, as the hardware does), and check what the kernel's comments state:
the error bounds of the fits, the signed-zero conventions of atan2 on the axes, and that the bins
they select differ from the bins of the FP64 angles no more often than FP32 rounding does.  The
device's rsqrtf is replaced by the exact reciprocal square root, so the bounds are those of the
polynomials themselves."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1708_06142_gb300", "csrc", "ts_column_dev.cuh")
F = np.float32


def _coefficients(name):
    """Coefficients of the Horner chain in function `name`, highest degree first."""
    src = open(SRC).read()
    body = src[src.index(f"float {name}("):]
    body = body[:body.index("\n}\n")]
    chain = body[body.index("fmaf("):body.index(";", body.index("fmaf("))]
    vals = [float(v) for v in re.findall(r"-?\d+\.\d+(?:e-?\d+)?(?=f)", chain)]
    assert len(vals) >= 6, vals
    return [F(v) for v in vals]


def _fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def _horner(coef, x):
    """coef highest degree first: ((c_n x + c_{n-1}) x + ...) x + c_0, one rounding per step."""
    r = np.full(x.shape, coef[0], dtype=F)
    r = _fma(r, x, np.full(x.shape, coef[1], dtype=F))
    for c in coef[2:]:
        r = _fma(r, x, np.full(x.shape, c, dtype=F))
    return r


def col_acos(u):
    x = np.abs(u).astype(F)
    om = (F(1) - x).astype(F)
    q = _horner(_coefficients("col_acos"), x)
    root = (om * (F(1) / np.sqrt(np.maximum(om, F(1e-30))))).astype(F)
    a = (q * root).astype(F)
    return np.where(u < 0, (F(np.pi) - a).astype(F), a)


def col_phi(y, x):
    ax, ay = np.abs(x).astype(F), np.abs(y).astype(F)
    mx = np.maximum(ax, ay)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(mx > 0, (np.minimum(ax, ay) / mx).astype(F), F(0))
    s = (a * a).astype(F)
    p = (a * _horner(_coefficients("col_phi"), s)).astype(F)
    p = np.where(ay > ax, (F(0.5 * np.pi) - p).astype(F), p)
    p = np.where(np.signbit(x), (F(np.pi) - p).astype(F), p)
    p = np.where(y < 0, (F(2 * np.pi) - p).astype(F), p)
    return p


def test_fit_error_bounds():
    x = np.linspace(0, 1, 2_000_001).astype(F)   # the fit's interval
    e_acos = np.abs(col_acos(x).astype(np.float64) - np.arccos(x.astype(np.float64))).max()
    assert e_acos < 4.1e-7, e_acos
    x = -x   # u < 0 through pi - acos|u|, one more FP32 rounding (half an ulp of pi)
    e_neg = np.abs(col_acos(x).astype(np.float64) - np.arccos(x.astype(np.float64))).max()
    assert e_neg < 4.1e-7 + 1.2e-7, e_neg
    t = np.linspace(0, 2 * np.pi, 2_000_001, endpoint=False)
    y, xx = np.sin(t).astype(F), np.cos(t).astype(F)
    ref = np.mod(np.arctan2(y.astype(np.float64), xx.astype(np.float64)), 2 * np.pi)
    d = np.abs(col_phi(y, xx).astype(np.float64) - ref)
    d = np.minimum(d, 2 * np.pi - d)   # 0 and 2 pi are the same direction
    # the fit, the rounding of min/max, and one rounding for each of the three identities
    # (pi/2 - p, pi - p, 2 pi - p: half an ulp of pi/2, pi and 2 pi)
    assert d.max() < 1.4e-7 + 0.6e-7 + 0.6e-7 + 1.2e-7 + 2.4e-7, d.max()


def test_axis_conventions():
    z = F(0)
    nz = F(-0.0)
    # phi on the axes follows atan2's signed zeros, wrapped to [0, 2 pi)
    got = col_phi(np.array([z, nz, z, nz, F(1), F(-1), z, z], F), np.array([F(1), F(1), F(-1), F(-1), z, z, nz, z], F))
    want = np.array([0, 0, np.pi, np.pi, np.pi / 2, 3 * np.pi / 2, np.pi, 0], np.float32)
    np.testing.assert_allclose(got, want, atol=2e-7)
    # theta at the poles and the equator
    np.testing.assert_allclose(col_acos(np.array([1, -1, 0, nz], F)), [0, np.pi, np.pi / 2, np.pi / 2], atol=4e-7)


def test_bins_match_fp64_angles_as_often_as_fp32_rounding():
    nth, nph = 25, 50   # the default table's theta and phi bins
    rng = np.random.default_rng(11)
    n = 1_000_000
    d = rng.integers(-8, 9, size=(n, 3)).astype(F) * F(1 / 128)   # separations of leaf cells on a grid
    d[n // 2:] = (rng.standard_normal((n - n // 2, 3)) * 0.1).astype(F)
    d = d[np.any(d != 0, axis=1)]
    dx, dy, dz = d[:, 0], d[:, 1], d[:, 2]
    inv = (F(1) / np.sqrt((dx * dx + dy * dy + dz * dz).astype(F))).astype(F)
    uz = np.clip(-dz * inv, F(-1), F(1)).astype(F)
    clamp = lambda v, m: np.clip(np.floor(v), 0, m - 1)
    it = clamp((col_acos(uz) * F(1 / np.pi) * F(nth)).astype(F), nth)
    ip = clamp((col_phi(-dy, -dx) * F(0.5 / np.pi) * F(nph)).astype(F), nph)
    D = d.astype(np.float64)
    r = np.sqrt((D ** 2).sum(1))
    th = np.arccos(np.clip(-D[:, 2] / r, -1, 1))
    ph = np.mod(np.arctan2(-D[:, 1], -D[:, 0]), 2 * np.pi)
    ph = np.where((D[:, 0] == 0) & (D[:, 1] == 0), np.pi, ph)   # along z: phi from -0 x-component
    it64, ip64 = clamp(th / np.pi * nth, nth), clamp(ph / (2 * np.pi) * nph, nph)
    # FP32 rounding of the same directions alone (exact angles of the FP32 unit vector)
    assert np.mean(it != it64) < 1e-5 and np.mean(ip != ip64) < 1e-5, (np.sum(it != it64), np.sum(ip != ip64))
