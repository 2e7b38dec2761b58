"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/lts.h declares.  No compute call: this runs without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "lts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lts_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_00083_gb300 import build as libbuild

    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    assert declared_entry_points() == sorted(
        ["lts_create", "lts_workspace_bytes", "lts_simplify", "lts_last_error", "lts_destroy",
         "lts_order_field_static", "lts_simplify_batch", "lts_submit", "lts_poll", "lts_simplify_persistence",
         "lts_serve_config", "lts_simplify_f64", "lts_classify", "lts_set_tuning", "lts_get_tuning"])


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_argument_checks_need_no_device(lib):
    import paper_2009_00083_gb300 as lts

    lts.load()
    ctx = ctypes.c_void_p()
    # invalid sizes are rejected before any CUDA call
    assert lts.load().lts_create(ctypes.byref(ctx), 0, 2, None) == 1
    assert lts.load().lts_create(ctypes.byref(ctx), 0, 1 << 31, None) == 1
    assert lts.load().lts_create(None, 0, 100, None) == 1
    g = lts.grid_of_shape((4, 5))
    assert lts.lts_workspace_bytes(g) > 0
    bad = lts.LtsGrid()
    bad.ndim = 4
    assert lts.lts_workspace_bytes(bad) == 0
    assert lts.load().lts_simplify(None, ctypes.byref(g), None, None, 0, 3, None, None, None) == 1
    assert lts.load().lts_simplify_persistence(None, ctypes.byref(g), None, 0.5, 3, None, None, None) == 1
    assert lts.load().lts_simplify_batch(None, 1, None, None, None, None, 3, None, None, None) == 1
    assert lts.load().lts_submit(None, ctypes.byref(g), None, None, 0, 3, None, None, None) == 1
    assert lts.load().lts_poll(None, 1, None) == 1
    assert lts.load().lts_simplify_f64(None, ctypes.byref(g), None, None, 0, 3, None, None, None) == 1
    assert lts.load().lts_classify(None, ctypes.byref(g), None, None, None, None) == 1
    assert lts.load().lts_set_tuning(None, None) == 1
    assert lts.load().lts_get_tuning(None, None) == 1


def test_static_order_field_rejects_oversize_grids_before_any_device_call(lib):
    import paper_2009_00083_gb300 as lts

    assert lts.ORDER_STATIC_MAX_VERTICES == 1 << 20
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape((1025, 1024)), 16, 1 << 40)
    assert code == 1 and "at most 1048576" in msg, msg
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape((65, 128, 128)), 16, 1 << 40)
    assert code == 1 and "1064960 vertices" in msg, msg
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape((8, 8)), 0, 1 << 40)
    assert code == 1 and "null" in msg
    code, msg = lts.lts_order_field_static(0, lts.grid_of_shape((8, 8)), 1 << 40, (1 << 40) + 128)
    assert code == 1 and "overlaps" in msg
    bad = lts.LtsGrid()
    bad.ndim = 3
    assert lts.lts_order_field_static(0, bad, 16, 1 << 40)[0] == 1
