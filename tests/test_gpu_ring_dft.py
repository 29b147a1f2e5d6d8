"""The ring-DFT stages alone (sht_ring_analysis / sht_ring_synthesis) against the oracle's direct
O(N^2) DFT sums (oracle/ring.py), element by element: every ring at band-limits that cover the
direct rings (k <= 31), the chirp-z classes and their boundaries (lengths 2^a and 3 2^a), and
sampled rings of every class at L = 1024 with 64 signals (the benchmark's launch configuration) and
at L = 2048 (the longest ring, 4095 samples, chirp-z length 8192).  Float64 and float32 plans.

Tolerance, from the arithmetic: a length-M FFT of a vector x errs by at most about
c u log2(M) ||x||_2 in the 2-norm (u the unit roundoff); the chirp-z form takes three such FFTs
of length M <= 4N.  Per ring the 2-norm of the error bounds every element, so the bins (1/N
scaled, ||B_k||_2 = ||s_k||_2 / sqrt(N)) are compared within 32 u (log2(4N) + 1) ||s_k||_2 / sqrt(N)
and the synthesised samples (||s_k||_2 = sqrt(N) ||B_k||_2) within 32 u (log2(4N) + 1) ||B_k||_2
sqrt(N).
"""
import math

import numpy as np
import pytest
import torch

from oracle import ring as oring
from paper_1403_4661_gb300 import synth
from tests.helpers import oracle_thetas

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1403_4661_gb300 import build
    build.build()


def _plan(L, dtype, keep_ptilde=True):
    from paper_1403_4661_gb300.sht import Plan
    return Plan(L, theta=oracle_thetas(L), dtype=dtype, keep_ptilde=keep_ptilde)


def _tol(u, k, norm):
    N = 2 * k + 1
    return 32.0 * u * (math.log2(4 * N) + 1.0) * norm / math.sqrt(N)


def _check_rings(L, dtype, s, bins_gpu, s2_gpu, rows, rings):
    """Compare GPU bins and synthesised samples of signals `rows` on `rings` with the oracle."""
    u = U[dtype]
    ref_b = oring.ring_dft(s[rows], L, rings)
    ref_s = oring.ring_idft(bins_gpu[rows], L, rings)     # the oracle's synthesis of the GPU bins
    for i, r in enumerate(rows):
        for k in rings:
            N = 2 * k + 1
            sl = slice(k * k, k * k + N)
            tb = _tol(u, k, np.linalg.norm(s[r, sl]))
            assert np.abs(bins_gpu[r, sl] - ref_b[i, sl]).max() <= tb, (L, dtype, r, k)
            ts = _tol(u, k, np.linalg.norm(bins_gpu[r, sl])) * N
            assert np.abs(s2_gpu[r, sl] - ref_s[i, sl]).max() <= ts, (L, dtype, r, k)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("L", [1, 2, 31, 33, 100, 300])
def test_every_ring_against_direct_dft(L, dtype):
    p = _plan(L, dtype)
    B = 3
    s = synth.uniform_samples(L, B, 40 + L)
    ct = torch.complex64 if dtype == "f32" else torch.complex128
    x = torch.from_numpy(s).to(DEV).to(ct)
    bins = p.ring_analysis(x)
    s2 = p.ring_synthesis(bins)
    torch.cuda.synchronize()
    s_in = x.cpu().numpy().astype(np.complex128)
    _check_rings(L, dtype, s_in, bins.cpu().numpy().astype(np.complex128),
                 s2.cpu().numpy().astype(np.complex128), list(range(B)), list(range(L)))
    # the round trip closes up to the same bound (synthesis of the analysis)
    scale = float(np.abs(s_in).max()) if s_in.size else 1.0
    assert float((s2 - x).abs().max()) <= 64 * U[dtype] * (math.log2(8 * L) + 1) * max(1.0, scale) * math.sqrt(2 * L)


def _class_rings(L):
    """Rings at the boundaries of every chirp-z class below L (lengths 2^a, 3 2^a >= 2N - 1), the
    last direct ring and the top ring."""
    ks = {0, 1, 31, 32, L - 1}
    for a in range(6, 14):
        for M in (2 ** a, 3 * 2 ** (a - 1)):
            kmax = (M // 2 + 1) // 2 - 1          # largest k with 2(2k+1) - 1 <= M
            ks.update({kmax, kmax + 1})
    return sorted(k for k in ks if 0 <= k < L)


def test_full_size_launch_sampled_rings():
    """L = 1024, 64 signals (the benchmark's batch): the ring classes' boundary rings of the first
    and last signal."""
    L, B = 1024, 64
    p = _plan(L, "f64")
    s = synth.uniform_samples(L, B, 77)
    x = torch.from_numpy(s).to(DEV)
    bins = p.ring_analysis(x)
    s2 = p.ring_synthesis(bins)
    torch.cuda.synchronize()
    _check_rings(L, "f64", s, bins.cpu().numpy(), s2.cpu().numpy(), [0, B - 1], _class_rings(L))


def test_L2048_longest_rings():
    """L = 2048, one signal, on a plan without the P~ table: the longest rings (chirp-z length
    8192) and the class boundaries below them."""
    L = 2048
    p = _plan(L, "f64", keep_ptilde=False)
    s = synth.uniform_samples(L, 1, 91)
    x = torch.from_numpy(s).to(DEV)
    bins = p.ring_analysis(x)
    s2 = p.ring_synthesis(bins)
    torch.cuda.synchronize()
    rings = _class_rings(L) + [2046]
    _check_rings(L, "f64", s, bins.cpu().numpy(), s2.cpu().numpy(), [0], sorted(set(rings)))


def test_edge_cases():
    from paper_1403_4661_gb300.sht import SHTError
    p = _plan(8, "f64")
    x = torch.zeros((0, 64), dtype=torch.complex128, device=DEV)
    assert p.ring_analysis(x).shape == (0, 64)
    y = torch.zeros((2, 64), dtype=torch.complex128, device=DEV)
    with pytest.raises(SHTError, match="INVALID_ARG"):
        p.ring_analysis(y, out=y)                  # input and output overlap
