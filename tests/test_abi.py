"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; host-side argument checks work without a GPU (no kernel runs)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(pt_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1504_07433_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_status_strings(lib):
    lib.pt_version.restype = ctypes.c_int
    assert lib.pt_version() >= 100
    lib.pt_status_string.restype = ctypes.c_char_p
    assert lib.pt_status_string(0) == b"ok"
    assert b"argument" in lib.pt_status_string(1)


def test_host_side_argument_checks(lib):
    import paper_1504_07433_gb300 as pt
    L = pt.load_library()
    # null orbit -> PT_ERR_ARG, before any CUDA call
    assert L.pt_ma_quad(None, 10, None, None, 0, None, 1, 1, 0.0, 16, None, None, None, None, None, 0, None,
                        None) == 1
    o = pt.Orbit(None, None, None, None, None, None, 4)
    # missing arrays
    assert L.pt_z_circ(None, 10, ctypes.byref(o), 1, 0.0, None, None) == 1
    # e without w
    o2 = pt.Orbit(1, 1, 1, 1, 1, None, 4)
    assert L.pt_z_circ(ctypes.c_void_p(8), 10, ctypes.byref(o2), 1, 0.0, ctypes.c_void_p(8), None) == 1
    # no outputs requested
    o3 = pt.Orbit(8, 8, 8, 8, None, None, 4)
    assert L.pt_ma_quad(ctypes.c_void_p(8), 10, ctypes.byref(o3), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), 1,
                        1, 0.0, 16, None, None, None, None, ctypes.c_void_p(8), 1 << 20, None, None) == 1
    # work buffer missing -> PT_ERR_WORKSPACE
    assert L.pt_ma_quad(ctypes.c_void_p(8), 10, ctypes.byref(o3), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), 1,
                        1, 0.0, 16, None, None, ctypes.c_void_p(8), None, None, 0, None, None) == 5
    # work buffer too small -> PT_ERR_WORKSPACE
    assert L.pt_ma_quad(ctypes.c_void_p(8), 10, ctypes.byref(o3), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), 1,
                        1, 0.0, 16, None, None, ctypes.c_void_p(8), None, ctypes.c_void_p(8), 16, None, None) == 5
    # supersampling out of range
    assert L.pt_ma_quad(ctypes.c_void_p(8), 10, ctypes.byref(o3), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), 1,
                        0, 0.0, 16, None, None, ctypes.c_void_p(8), None, ctypes.c_void_p(8), 1 << 20, None,
                        None) == 1
    # a negative or non-finite exposure time -> PT_ERR_DOMAIN, before any CUDA call
    for bad_exp in (-0.01, float("nan"), float("inf")):
        assert L.pt_ma_quad(ctypes.c_void_p(8), 10, ctypes.byref(o3), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), 1,
                            3, bad_exp, 16, None, None, ctypes.c_void_p(8), None, ctypes.c_void_p(8), 1 << 20, None,
                            None) == 2
        assert L.pt_z_circ(ctypes.c_void_p(8), 10, ctypes.byref(o3), 3, bad_exp, ctypes.c_void_p(8), None) == 2
    assert b"exposure" in L.pt_last_error_string()
    # domain check: a missing counter or radius-ratio array is an argument error
    assert L.pt_domain_check(ctypes.byref(o3), ctypes.c_void_p(8), 1, None, None) == 1
    assert L.pt_domain_check(ctypes.byref(o3), None, 1, ctypes.c_void_p(8), None) == 1
    assert L.pt_domain_check(ctypes.byref(o3), ctypes.c_void_p(8), 0, ctypes.c_void_p(8), None) == 1
    # Gimenez plan arguments are checked before allocation
    h = ctypes.c_void_p()
    assert L.pt_gim_plan_create(0, 100, ctypes.byref(h)) == 1
    assert L.pt_gim_plan_create(8, 1, ctypes.byref(h)) == 1


def test_work_bytes_grow_with_problem(lib):
    import paper_1504_07433_gb300 as pt
    a = pt.ma_quad_work_bytes(1000, 4, 1)
    b = pt.ma_quad_work_bytes(100000, 256, 1)
    c = pt.ma_quad_work_bytes(100000, 256, 4, k_per_band=True)
    assert 0 < a < b < c
