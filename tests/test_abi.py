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


def test_every_entry_point_refuses_a_null_plan_without_gpu(lib):
    """Each entry point that takes a plan answers SHT_ERR_INVALID_ARG (1) for NULL on the host."""
    P = ctypes.c_void_p
    n = None
    assert lib.sht_inverse(n, n, n, 1, n) == 1
    assert lib.sht_forward_adjoint(n, n, n, 1, n) == 1
    assert lib.sht_inverse_adjoint(n, n, n, 1, n) == 1
    assert lib.sht_forward_noalloc(n, n, n, 1, n) == 1
    assert lib.sht_plan_reserve(n, 1) == 1
    assert lib.sht_plan_set_refinement(n, 3, 1e-11) == 1
    assert lib.sht_plan_set_wait_limit(n, 1.0) == 1
    assert lib.sht_plan_set_timing(n, 1) == 1
    assert lib.sht_plan_stage_times(n, n, n) == 1
    assert lib.sht_plan_check(n) == 1
    assert lib.sht_plan_thetas(n, n) == 1
    assert lib.sht_get_info(n, n) == 1
    assert lib.sht_plan_bandlimit(n) == 0
    assert lib.sht_plan_destroy(n) == 0                               # NULL is a no-op
    assert lib.sht_plan_save(n, b"x") == 1
    h = P()
    assert lib.sht_plan_load(n, 0, ctypes.byref(h)) == 1
    assert lib.sht_plan_with_thetas(8, 0, n, 0, ctypes.byref(h)) == 1  # NULL co-latitudes
    bad = (ctypes.c_double * 8)(*([4.0] * 8))                          # outside [0, pi]
    assert lib.sht_plan_with_thetas(8, 0, bad, 0, ctypes.byref(h)) == 1
    assert lib.sht_plan_with_thetas(0, 0, bad, 0, ctypes.byref(h)) == 2
    # uneven calls: nothing to do, or a negative count
    assert lib.sht_forward_uneven(n, 0, 0, n, n, n, n, n) == 0
    assert lib.sht_inverse_uneven(n, 0, -1, n, n, n, n, n) == 1
    assert lib.sht_forward_uneven(n, 0, 3, n, n, n, n, n) == 1
