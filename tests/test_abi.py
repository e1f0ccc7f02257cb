"""The C-ABI library builds for sm_103a, loads on a machine without a GPU and
exports every entry point include/amg_b300.h declares.  No compute calls."""
import ctypes as C
import os
import re

import pytest

from paper_2606_09001_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amg_b300.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amg_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_loads():
    path = build.build()
    assert os.path.exists(path)
    _lib.load()


def test_every_declared_symbol_is_exported():
    L = _lib.load()
    decl = declared_functions()
    assert decl, "no declarations parsed"
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(_lib.EXPORTS)


def test_config_defaults_and_status_strings():
    L = _lib.load()
    c = _lib.AmgConfig()
    assert L.amg_config_default(C.byref(c)) == 0
    assert c.solver == 0 and c.omega == pytest.approx(2 / 3) and c.theta == 0.08
    assert c.coarse_max == 64 and c.rtol == 1e-8 and c.precision == 0 and c.symmetric == -1
    assert c.layout == 0 and c.adjoint_reuse == 0 and c.amg_type == 0 and c.fuse_coarse == 1
    assert c.device_loop == 1 and c.outer_product == -1
    assert L.amg_config_default(None) == _lib.AMG_ERR_ARG
    for code in (0, 1, 2, 3, 4, -1, -2, -3, -4, -5, -6, -7):
        assert _lib.status_string(code) != "unknown status"


def test_argument_errors_need_no_device():
    L = _lib.load()
    h = C.c_void_p()
    # n <= 0 and null arrays are rejected before any CUDA call
    assert L.amg_setup(None, 0, 0, None, None, None, None, C.byref(h)) == _lib.AMG_ERR_ARG
    assert L.amg_setup(None, 4, 4, None, None, None, None, C.byref(h)) == _lib.AMG_ERR_ARG
    assert L.amg_setup(None, 4, 4, None, None, None, None, None) == _lib.AMG_ERR_ARG
    assert h.value is None
    assert L.amg_solve(None, None, None, None, None) == _lib.AMG_ERR_ARG
    assert L.amg_adjoint(None, None, None, None, None, None, None) == _lib.AMG_ERR_ARG
    assert L.amg_free(None) == 0


def test_config_struct_layout_matches_header():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    structs = {name: body for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+);", src, re.S)}
    for cname, ctype in (("amg_config", _lib.AmgConfig), ("amg_info", _lib.AmgInfo)):
        names = re.findall(r"\b(\w+)\s*(?:\[\w+\])?\s*[;,]", structs[cname])
        assert names == [f for f, _ in ctype._fields_], cname
