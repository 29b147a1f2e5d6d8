"""The C-ABI library: it builds, loads, exports every function include/sht.h declares, and its
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(sht_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1403_4661_gb300 import build, sht
    build.build()
    return sht.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "sht_forward" in names and "sht_inverse" in names and len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1403_4661_gb300 import sht
    assert sorted(sht.EXPORTED) == sorted(n for n in _declared())


def test_host_argument_checks_without_gpu(lib):
    h = ctypes.c_void_p(1)
    assert lib.sht_plan(0, 0, 0, ctypes.byref(h)) == 2          # SHT_ERR_UNSUPPORTED
    assert h.value is None
    assert lib.sht_plan(5000, 0, 0, ctypes.byref(h)) == 2
    assert lib.sht_plan(8, 6, 0, ctypes.byref(h)) == 2           # unknown dtype
    assert lib.sht_plan(8, -1, 0, ctypes.byref(h)) == 2
    assert lib.sht_plan(8, 0, 0, None) == 1                      # SHT_ERR_INVALID_ARG
    assert lib.sht_plan(8, 0, 6, ctypes.byref(h)) == 1           # both ring-measure bits
    assert lib.sht_forward(None, None, None, 1, None) == 1       # NULL plan
    assert lib.sht_plan_set_paths(None, 1, 0, 0, 0) == 1
    assert lib.sht_plan_autotune(None, 1, None) == 1
    assert lib.sht_status_string(4) == b"SHT_ERR_CUDA"
    assert b"plan" in lib.sht_last_error_message() or lib.sht_last_error_message() != b""
