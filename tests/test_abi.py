"""The C-ABI library builds, loads and exports every symbol include/fnt_rs.h declares.

CPU-only: no compute call is made (there may be no GPU here).
"""
import ctypes
import re

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_0907_1788_gb300 import build, _lib

    build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_symbols_exported(lib):
    from paper_0907_1788_gb300 import _lib

    names = _lib.declared_symbols()
    assert "fnt_rs_encode" in names and "fnt_rs_decode" in names and "fnt_rs_plan_create" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/fnt_rs.h but not exported"


def test_binding_names_match_header():
    import paper_0907_1788_gb300 as pkg
    from paper_0907_1788_gb300 import _lib

    for name in _lib.declared_symbols():
        assert hasattr(pkg, name), f"binding lacks {name}"


def test_strerror_without_gpu():
    import paper_0907_1788_gb300 as pkg

    assert pkg.fnt_rs_strerror(0) == "ok"
    assert "65537" in pkg.fnt_rs_strerror(-2)
    assert "debug build" in pkg.fnt_rs_strerror(pkg.E_BOUNDS)


def test_release_build_has_no_device_index_checks(lib):
    # the checks of the debug build (-DFNTRS_DEBUG_BOUNDS=1) are compiled out here
    assert lib.fnt_rs_debug_bounds() == 0


def test_argument_errors_without_gpu():
    # validation happens on the host before any CUDA call
    import paper_0907_1788_gb300 as pkg

    lib = pkg.load()
    h = ctypes.c_void_p()
    assert lib.fnt_rs_plan_create(ctypes.byref(h), 12, 4, 65537, 0, None) == -1  # n not 2^i
    assert lib.fnt_rs_plan_create(ctypes.byref(h), 16, 17, 65537, 0, None) == -1  # k > n
    assert lib.fnt_rs_plan_create(ctypes.byref(h), 16, 0, 65537, 0, None) == -1  # k = 0
    assert lib.fnt_rs_plan_create(ctypes.byref(h), 16, 8, 257, 0, None) == -2  # p
    assert lib.fnt_rs_plan_create(ctypes.byref(h), 16, 8, 65537, 3, None) == -3  # order 65536
    assert lib.fnt_rs_plan_create(ctypes.byref(h), 1 << 17, 8, 65537, 0, None) == -1
    assert lib.fnt_rs_encode(None, None, 0, None, 0, 4, None, None) == -1


def test_header_cites_paper_for_every_entry_point():
    import os

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "fnt_rs.h")).read()
    assert re.search(r"Sec\. II\.B", hdr)
    for name in ["fnt_rs_encode", "fnt_rs_decode_prepare", "fnt_rs_decode", "fnt_rs_fnt"]:
        block = hdr[: hdr.index(name + "(")].rsplit("/*", 1)[1]
        assert "Sec." in block, f"{name} comment lacks a citation"
