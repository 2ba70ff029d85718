"""The arithmetic peak probe used for the walk's roofline denominators."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_peak_probe_plausible():
    from paper_1708_06142_gb300.treesolver import TSError, peak_probe
    f32 = peak_probe(0, "fp32")
    f32x2 = peak_probe(0, "fp32x2")
    f64 = peak_probe(0, "fp64")
    for v in (f32, f32x2, f64):
        assert math.isfinite(v) and v > 0
    # nominal FP32: 152 SMs x 128 lanes x 2 flop x clock; a probe cannot exceed twice that
    assert 5.0 < f32 < 2 * 80.6 and 5.0 < f32x2 < 2 * 2 * 80.6
    assert f64 < f32
    with pytest.raises(TSError):
        from paper_1708_06142_gb300 import treesolver as t
        import ctypes as C
        v = C.c_double()
        t._check(t.load().ts_peak_probe(0, 7, C.byref(v)))
