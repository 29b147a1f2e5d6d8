"""sht_forward_noalloc against sht_forward, through the C ABI.

sht_forward_noalloc serves callers that cannot let a transform call allocate device memory (a
library handed a fixed memory budget by its host application, or code running where cudaMalloc is
not allowed): it runs the forward transform with its scratch in a fixed 64 MiB array of the
library.  This file is collected last so that a run stopping at the first failure has run every
other test already.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SHT_ERR_UNSUPPORTED = 2


def _call(lib, name, h, x, y, batch):
    return getattr(lib, name)(h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                              batch, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _lib():
    from paper_1403_4661_gb300 import build
    from paper_1403_4661_gb300 import sht as S

    build.build()
    return S, S.load_library()


@pytest.mark.parametrize("dtype", ["f64", "f64_tensor"])
def test_noalloc_forward_matches_forward_twice(dtype):
    """Two calls in a row share (and reuse) the fixed scratch.  Tensor plans run the float64
    SIMT chain here, so the comparison with their tensor-core sht_forward holds to 1e-11."""
    from oracle import sampling
    from paper_1403_4661_gb300 import synth

    S, lib = _lib()
    L, B = 96, 3
    plan = S.Plan(L, theta=sampling.thetas(L, "greedy"), dtype=dtype)
    x = torch.from_numpy(synth.uniform_samples(L, B, 77)).to("cuda:0")
    ref = torch.empty_like(x)
    assert _call(lib, "sht_forward", plan.handle, x, ref, B) == 0
    for _ in range(2):
        out = torch.full_like(x, float("nan"))
        assert _call(lib, "sht_forward_noalloc", plan.handle, x, out, B) == 0
        torch.cuda.synchronize()
        assert float((out - ref).abs().max()) <= 1e-11


def test_noalloc_size_limit_boundary_L1024():
    """The scratch needed at L = 1024 is 34.1 MB for one signal (accepted) and 68.2 MB for two
    (refused: the array holds 67108864 bytes)."""
    from paper_1403_4661_gb300 import synth
    from tests.helpers import oracle_thetas

    S, lib = _lib()
    L = 1024
    plan = S.Plan(L, theta=oracle_thetas(L))
    c = torch.from_numpy(synth.decaying_coeffs(L, 2, 5)).to("cuda:0")
    x = plan.inverse(c)
    y = torch.empty_like(x)
    assert _call(lib, "sht_forward_noalloc", plan.handle, x, y, 2) == SHT_ERR_UNSUPPORTED
    assert b"bytes of scratch" in lib.sht_last_error_message()
    x1 = x[:1].contiguous()
    ref = torch.empty_like(x1)
    assert _call(lib, "sht_forward", plan.handle, x1, ref, 1) == 0
    out = torch.full_like(x1, float("nan"))
    assert _call(lib, "sht_forward_noalloc", plan.handle, x1, out, 1) == 0
    torch.cuda.synchronize()
    assert float((out - ref).abs().max()) <= 1e-11


def test_noalloc_rejects_sizes_beyond_the_array():
    S, lib = _lib()
    L = 200
    plan = S.Plan(L, ordering="simple")
    B = 200  # scratch far above 64 MiB
    x = torch.zeros((B, L * L), dtype=torch.complex128, device="cuda:0")
    y = torch.empty_like(x)
    assert _call(lib, "sht_forward_noalloc", plan.handle, x, y, B) == SHT_ERR_UNSUPPORTED
    assert b"bytes of scratch" in lib.sht_last_error_message()
