"""The C-ABI library builds, loads and exports every entry point that include/tt.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tt_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._load_builder().build()


def test_every_declared_symbol_is_exported(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert "tt_forward" in names and "tt_adjoint" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi(lib_path):
    import paper_2412_00031_gb300 as tt
    for n in declared_functions():
        assert n in tt.EXPORTED


def test_default_opts_and_struct_layout(lib_path):
    import paper_2412_00031_gb300 as tt
    o = tt.default_opts(tt.TT_F32)
    assert o.tol_fwd == pytest.approx(1e-6) and o.max_iter_fwd == 500 and o.launch_blocks == 0
    o = tt.default_opts(tt.TT_F64)
    assert o.tol_fwd == pytest.approx(1e-8)
    # host-side structs mirror the C layout
    assert ctypes.sizeof(tt.TTPoint) == 24
    assert ctypes.sizeof(tt.TTGrid) == 4 * 3 + 4 + 8 * 7 + 8


def test_invalid_grid_rejected_without_device_work(lib_path):
    import paper_2412_00031_gb300 as tt
    h = ctypes.c_void_p()
    g = tt.TTGrid(3, 10, 10, 0.0, 10.0, 0.0, 1.0, 0.0, 1.0, 6371.0, 0)  # n_r < 4
    assert tt.lib.tt_ctx_create(ctypes.byref(h), ctypes.byref(g), None) == tt.TT_EINVAL
    g = tt.TTGrid(10, 10, 10, 10.0, 0.0, 0.0, 1.0, 0.0, 1.0, 6371.0, 0)  # depth range reversed
    assert tt.lib.tt_ctx_create(ctypes.byref(h), ctypes.byref(g), None) == tt.TT_EINVAL
    g = tt.TTGrid(10, 10, 10, 0.0, 10.0, 0.0, 1.0, 0.0, 1.0, 6371.0, 7)  # unknown geometry
    assert tt.lib.tt_ctx_create(ctypes.byref(h), ctypes.byref(g), None) == tt.TT_EINVAL
