"""The C-ABI library: loads without a GPU and exports every entry point include/*.h declares."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^TS_API\s+[\w\s\*]+?\b(ts_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("ts_create", "ts_destroy", "ts_tree_build", "ts_ewald_field", "ts_gravity_walk", "ts_column_walk",
              "ts_sync"):
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_1708_06142_gb300 import treesolver as ts
    L = ts.load(build_if_missing=True)
    names = declared_symbols()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(L, n), f"{n} not exported"
        assert n in ts.SIGNATURES, f"{n} has no binding"
    assert set(ts.SIGNATURES) == names
    assert ts.version().startswith("treesolver-gb300")


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1708_06142_gb300 import treesolver as ts
    with pytest.raises(ts.TSError) as e:
        ts.TreeSolver(0)
    assert e.value.status in (1, 4)


def test_struct_layouts_match_header():
    # the binding's ctypes structures must have the C layout the header implies (x86_64 / aarch64 LP64)
    import ctypes as C
    from paper_1708_06142_gb300 import treesolver as ts
    assert C.sizeof(ts.TSMesh) == 4 + 4 + 8 * 4 + 12 + 4
    assert ts.TSGravityParams.theta.offset == 8 and ts.TSGravityParams.a_old_dev.offset == 32
    assert C.sizeof(ts.TSGravityParams) == 80
    assert C.sizeof(ts.TSColumnParams) == 64
    assert C.sizeof(ts.TSShieldParams) == 80 and ts.TSShieldParams.co_table.offset == 40
    assert ts.TSGravityParams.accel.offset == 68
