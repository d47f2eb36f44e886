"""The C ABI library (no GPU needed): it builds, loads, exports every function include/bcg.h declares,
and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libbcg():
    from paper_1912_11930_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(bcg_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(libbcg):
    names = _declared()
    assert {"bcg_create_csr", "bcg_create_stencil", "bcg_solve", "bcg_destroy"} <= set(names)
    missing = [n for n in names if not hasattr(libbcg, n)]
    assert not missing, missing


def test_host_side_argument_errors(libbcg):
    vp = ctypes.c_void_p
    libbcg.bcg_create_csr.restype = ctypes.c_int
    libbcg.bcg_create_csr.argtypes = [ctypes.POINTER(vp), ctypes.c_int64, ctypes.c_int64, vp, vp, vp,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp]
    libbcg.bcg_last_error.restype = ctypes.c_char_p
    h = vp()
    assert libbcg.bcg_create_csr(ctypes.byref(h), 0, 1, None, None, None, 4, 2, 0, 0, None) == 1
    assert b"n=0" in libbcg.bcg_last_error()
    assert libbcg.bcg_create_csr(ctypes.byref(h), 10, 10, None, None, None, 6, 4, 0, 0, None) == 1
    assert b"divide" in libbcg.bcg_last_error()
    assert libbcg.bcg_create_csr(ctypes.byref(h), 10, 10, None, None, None, 4, 2, 9, 0, None) == 1
    assert libbcg.bcg_create_csr(None, 10, 10, None, None, None, 4, 2, 0, 0, None) == 1
    libbcg.bcg_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_double]
    assert libbcg.bcg_set_option(None, b"graph", 1.0) == 1
    libbcg.bcg_destroy.argtypes = [vp]
    libbcg.bcg_destroy(None)   # NULL-safe
