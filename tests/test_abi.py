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
    return sorted(set(re.findall(r"\b(lts_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_00083_gb300 import build as libbuild

    path = libbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    assert declared_entry_points() == sorted(
        ["lts_create", "lts_workspace_bytes", "lts_simplify", "lts_last_error", "lts_destroy"])


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
