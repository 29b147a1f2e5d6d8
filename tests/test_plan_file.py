"""Co-latitude files of sht_plan_save / sht_plan_load: the loader checks a file before any device
work.  Files are written here from the format's definition in include/sht.h: the tag "SHTTHETA",
int32 L, int32 0, L float64 values, then the 64-bit FNV-1a hash (offset basis 0xcbf29ce484222325,
prime 0x100000001b3) of everything before it."""
import ctypes
import math
import struct

import numpy as np
import pytest

SHT_ERR_INVALID_ARG = 1


def fnv1a64(data):
    h = 0xCBF29CE484222325
    for byte in data:
        h ^= byte
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def theta_file(L, thetas, tag=b"SHTTHETA", pad=0):
    body = tag + struct.pack("<ii", L, pad) + np.asarray(thetas, dtype="<f8").tobytes()
    return body + struct.pack("<Q", fnv1a64(body))


@pytest.fixture(scope="module")
def lib():
    from paper_1403_4661_gb300 import build, sht
    build.build()
    return sht.load_library()


def _load(lib, path):
    h = ctypes.c_void_p()
    st = lib.sht_plan_load(str(path).encode(), 0, ctypes.byref(h))
    return st, h


def test_fnv1a_reference_values():
    # published test vectors of 64-bit FNV-1a
    assert fnv1a64(b"") == 0xCBF29CE484222325
    assert fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert fnv1a64(b"foobar") == 0x85944171F73967E8


def test_damaged_files_are_rejected_before_device_work(lib, tmp_path):
    L = 6
    th = math.pi * (2.0 * np.arange(L) + 1.0) / (2.0 * L - 1.0)
    good = theta_file(L, th)
    cases = {
        "tag": theta_file(L, th, tag=b"SHTTHETB"),
        "pad": theta_file(L, th, pad=1),
        "L0": theta_file(0, []),
        "Lbig": theta_file(4096, np.zeros(4096)),
        "short": good[:-9],
        "long": good + b"\0",
        "flipped": good[:20] + bytes([good[20] ^ 1]) + good[21:],
        "empty": b"",
    }
    for name, data in cases.items():
        f = tmp_path / f"{name}.bin"
        f.write_bytes(data)
        st, h = _load(lib, f)
        assert st == SHT_ERR_INVALID_ARG, name
        assert h.value is None
    st, _ = _load(lib, tmp_path / "missing.bin")
    assert st == SHT_ERR_INVALID_ARG


def test_valid_file_passes_the_checks(lib, tmp_path):
    """A valid file gets past the checks: without a GPU the plan build itself then fails with
    SHT_ERR_CUDA (4); with one, the plan is built (and destroyed here)."""
    L = 6
    th = math.pi * (2.0 * np.arange(L) + 1.0) / (2.0 * L - 1.0)
    f = tmp_path / "ok.bin"
    f.write_bytes(theta_file(L, th[::-1]))
    st, h = _load(lib, f)
    assert st in (0, 4)
    if st == 0:
        lib.sht_plan_destroy(h)
    assert lib.sht_plan_save(None, str(f).encode()) == SHT_ERR_INVALID_ARG
