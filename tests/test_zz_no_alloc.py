"""sht_forward_noalloc against sht_forward, through the C ABI.

sht_forward_noalloc serves callers that cannot let a transform call allocate device memory: it
runs the forward transform with its scratch in a fixed 64 MiB array of the library.  This file is
collected last so that a run stopping at the first failure has run every other test already.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _call(lib, name, h, x, y, batch):
    return getattr(lib, name)(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                              batch, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_forward_matches_forward_twice():
    from oracle import sampling
    from paper_1403_4661_gb300 import build, synth
    from paper_1403_4661_gb300 import sht as S

    build.build()
    lib = S.load_library()
    L, B = 96, 3
    plan = S.Plan(L, theta=sampling.thetas(L, "greedy"))
    x = torch.from_numpy(synth.uniform_samples(L, B, 77)).to("cuda:0")
    ref = torch.empty_like(x)
    assert _call(lib, "sht_forward", plan.handle, x, ref, B) == 0
    for _ in range(2):  # two calls in a row share (and reuse) the fixed scratch
        out = torch.full_like(x, float("nan"))
        assert _call(lib, "sht_forward_noalloc", plan.handle, x, out, B) == 0
        torch.cuda.synchronize()
        assert float((out - ref).abs().max()) <= 1e-11


def test_noalloc_rejects_sizes_beyond_the_array():
    from paper_1403_4661_gb300 import build
    from paper_1403_4661_gb300 import sht as S

    build.build()
    lib = S.load_library()
    L = 200
    plan = S.Plan(L, ordering="simple")
    B = 200  # scratch far above 64 MiB
    x = torch.zeros((B, L * L), dtype=torch.complex128, device="cuda:0")
    y = torch.empty_like(x)
    assert _call(lib, "sht_forward_noalloc", plan.handle, x, y, B) == 2  # SHT_ERR_UNSUPPORTED
    assert b"64 MiB" in lib.sht_last_error_message() or b"bytes of scratch" in lib.sht_last_error_message()
