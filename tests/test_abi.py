"""CPU-only checks of the C ABI: the library loads, exports every function
include/dpg.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dpg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dpg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_cs_0308004_gb300 import _build
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dpg_retrieve", "dpg_retrieve_direct", "dpg_sort_copy", "dpg_sync", "dpg_ctx_create"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in dpg.h but not exported"


def test_binding_covers_the_header():
    from paper_cs_0308004_gb300 import dpg
    assert set(declared_functions()) <= set(dpg.SIGNATURES)


def test_host_side_argument_errors(lib):
    lib.dpg_strerror.restype = ctypes.c_char_p
    assert lib.dpg_strerror(0) == b"ok"
    assert lib.dpg_strerror(2) == b"rid or key out of range"
    f = lib.dpg_retrieve
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t, ctypes.c_size_t,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    # a null context is rejected before anything touches a device
    assert f(None, 16, 10, 4, 10, 32, 64, None) == 1
    lib.dpg_sync.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.dpg_sync(None, None) == 1
    lib.dpg_ctx_create.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.dpg_ctx_create(None, 0) == 1
    # failure-detection hooks refuse a null context on the host as well
    lib.dpg_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_double]
    assert lib.dpg_set_wait_limit(None, 1.0) == 1
    lib.dpg_check_wait.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.dpg_check_wait(None, None) == 1
    lib.dpg_inject_alloc_failure.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.dpg_inject_alloc_failure(None, 1) == 1
