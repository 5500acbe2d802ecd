"""The C ABI library builds, loads and exports every symbol its header declares.

No GPU needed: loading the library and calling the pure host functions
(status strings, supported lengths, argument validation that fails before any
CUDA call) works without a device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"CUBIC_API\s+[\w\s\*]*?\b(cubic_\w+)\s*\(", text)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2510_14143_gb300 import build
    return build.build()


def test_header_declares_the_abi():
    names = declared_symbols()
    for required in ("cubic_rl_plan", "cubic_rl_deconvolve", "cubic_rl_plan_destroy", "cubic_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi(libpath):
    import paper_2510_14143_gb300 as cr
    for n in declared_symbols():
        assert hasattr(cr, n), f"binding lacks {n}"


def test_host_only_calls(libpath):
    import paper_2510_14143_gb300 as cr
    assert cr.cubic_status_string(0) == "ok"
    assert cr.cubic_status_string(2) == "unsupported size"
    for n in (1, 2, 3, 5, 48, 75, 81, 125, 128, 160, 1024):
        assert cr.cubic_rl_supported_length(n), n
    for n in (0, 7, 11, 13, 97, 2049):
        assert not cr.cubic_rl_supported_length(n), n


def test_invalid_arguments_fail_before_any_launch(libpath):
    lib = ctypes.CDLL(libpath)
    lib.cubic_rl_plan.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.c_void_p, ctypes.c_uint, ctypes.c_void_p]
    lib.cubic_rl_deconvolve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_float,
                                        ctypes.c_void_p, ctypes.c_void_p]
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 7)             # 7 is not 5-smooth
    assert lib.cubic_rl_plan(ctypes.byref(h), dims, ctypes.c_void_p(256), 0, None) == 2
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    assert lib.cubic_rl_plan(ctypes.byref(h), dims, None, 0, None) == 1
    assert lib.cubic_rl_plan(ctypes.byref(h), dims, ctypes.c_void_p(258), 0, None) == 3
    assert lib.cubic_rl_plan(ctypes.byref(h), dims, ctypes.c_void_p(256), 1, None) == 1
    assert lib.cubic_rl_deconvolve(None, ctypes.c_void_p(256), 1, 1e-6, ctypes.c_void_p(512), None) == 1
    lib.cubic_rl_plan_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    assert lib.cubic_rl_plan_set_wait_limit(None, 1) == 1
