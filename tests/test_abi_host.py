"""Host-side checks of the C ABI that need no GPU.

The library must build, load and export every entry point that
include/bdct.h declares; argument validation that happens before any CUDA
call must return the documented status codes.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bdct_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared_symbols()
    for must in ("bdct_plan_create", "bdct_forward", "bdct_inverse", "bdct_roundtrip",
                 "bdct_plan_destroy", "bdct_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(bdct_lib):
    from paper_2609_28519_gb300 import native
    for name in _declared_symbols():
        assert hasattr(bdct_lib, name), name
    assert sorted(native.EXPORTS) == _declared_symbols()


def test_status_strings(bdct_lib):
    for s in range(0, 11):
        assert bdct_lib.bdct_status_string(s)
    assert bdct_lib.bdct_status_string(999) == b"unknown status"
    assert bdct_lib.bdct_version() >= 100


def test_argument_validation_before_cuda(bdct_lib):
    L = bdct_lib
    h = ctypes.c_void_p()
    assert L.bdct_plan_create(None, 8, 8, 1, 0, 0) == 1
    assert L.bdct_plan_create(ctypes.byref(h), 0, 8, 1, 0, 0) == 1
    assert L.bdct_plan_create(ctypes.byref(h), 8, -3, 1, 0, 0) == 1
    assert L.bdct_plan_create(ctypes.byref(h), 8, 8, 0, 0, 0) == 1
    assert L.bdct_plan_create(ctypes.byref(h), 8, 8, 16, 0, 0) == 1  # not a kind bit
    assert L.bdct_plan_create(ctypes.byref(h), 8, 8, 1, 7, 0) == 1
    assert L.bdct_plan_create(ctypes.byref(h), 8, 8, 1, 0, 9) == 1
    assert L.bdct_plan_create(ctypes.byref(h), 8, 10, 1, 0, 0) == 2  # cols not a multiple of 4
    assert L.bdct_plan_create(ctypes.byref(h), 16384, 8, 1, 0, 0) == 2
    assert h.value is None
    assert L.bdct_plan_destroy(None) == 0
    assert L.bdct_execute(None, 1, None, None, 1, None) == 1
    assert L.bdct_plan_set_spectral(None, None) == 1
    info = __import__("paper_2609_28519_gb300.native", fromlist=["PlanInfo"]).PlanInfo()
    assert L.bdct_plan_get_info(None, ctypes.byref(info)) == 1


def test_no_device_is_an_error_not_a_fallback(bdct_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("host has a GPU")
    h = ctypes.c_void_p()
    st = bdct_lib.bdct_plan_create(ctypes.byref(h), 8, 8, 1, 0, 0)
    assert st == 6  # BDCT_ERR_CUDA: no device, and no CPU fallback
    assert h.value is None
