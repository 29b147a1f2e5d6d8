"""Pins of the oracle's ring DFTs (oracle/ring.py): numpy's FFT of each ring (a library routine for
the same sum), the closed form of a single frequency, the round trip, Parseval's identity per ring,
and the alias relation of Eqs. (15) and (18): the bins of a band-limited signal's ring k are the
sums over the orders m = j (mod 2k+1) of G_m(theta_k) / 2 pi, with G_m of Eq. (11) built here from
the pinned P~ of oracle/legendre.py."""
import math

import numpy as np
import pytest

from oracle import legendre, ring, sampling, sht
from paper_1403_4661_gb300 import synth


@pytest.mark.parametrize("L", [1, 2, 5, 33])
def test_matches_numpy_fft_per_ring(L):
    s = synth.uniform_samples(L, 2, 3)
    bins = ring.ring_dft(s, L)
    for k in range(L):
        N = 2 * k + 1
        f = np.fft.fft(s[:, k * k:k * k + N], axis=1) / N
        for j in range(-k, k + 1):
            np.testing.assert_allclose(bins[:, k * k + k + j], f[:, j % N], atol=1e-15 * N, rtol=0)


def test_single_frequency_is_one_bin():
    L = 9
    for k in (0, 3, 8):
        N = 2 * k + 1
        for j0 in range(-k, k + 1):
            s = np.zeros(L * L, dtype=np.complex128)
            n = np.arange(N)
            s[k * k:k * k + N] = np.exp(2j * math.pi * j0 * n / N)
            bins = ring.ring_dft(s, L)
            want = np.zeros(L * L, dtype=np.complex128)
            want[k * k + k + j0] = 1.0
            np.testing.assert_allclose(bins, want, atol=1e-14)


@pytest.mark.parametrize("L", [1, 4, 40])
def test_round_trip_and_parseval(L):
    s = synth.uniform_samples(L, 3, 5)
    bins = ring.ring_dft(s, L)
    np.testing.assert_allclose(ring.ring_idft(bins, L), s, atol=1e-13, rtol=0)
    for k in range(L):
        N = 2 * k + 1
        e_s = np.sum(np.abs(s[:, k * k:k * k + N]) ** 2, axis=1)
        e_b = N * np.sum(np.abs(bins[:, k * k:k * k + N]) ** 2, axis=1)
        np.testing.assert_allclose(e_b, e_s, rtol=1e-13)


@pytest.mark.parametrize("L", [6, 17])
def test_bins_are_aliased_order_sums(L):
    th = sampling.thetas(L)
    c = synth.uniform_coeffs(L, 1, 8)[0]
    s = sht.inverse(c, L, th)
    bins = ring.ring_dft(s, L)
    want = np.zeros(L * L, dtype=np.complex128)
    for m in range(-(L - 1), L):
        am = abs(m)
        P = legendre.ptilde_order(am, L, th)                       # (L rings, L - |m|)
        sg = (-1.0) ** am if m < 0 else 1.0                        # Eq. (23)
        ell = np.arange(am, L)
        G = sg * (P @ c[ell * ell + ell + m])                      # G_m(theta_k) / 2 pi, Eq. (11)
        for k in range(L):
            N = 2 * k + 1
            j = (m + k) % N - k                                    # the bin order m aliases to
            want[k * k + k + j] += G[k]
    np.testing.assert_allclose(bins, want, atol=1e-13 * L, rtol=0)
