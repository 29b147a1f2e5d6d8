"""Ring DFTs of the optimal-dimensionality sampling by direct sums, plain float64.

Test infrastructure (oracle); see the package docstring.

Ring k (N_k = 2k+1 equispaced samples at phi_n = 2 pi n / N_k, Sec. III-A) enters Procedure 1
(Sec. III-C) through its DFT, the sum over phi of Eq. (11), and leaves Procedure 2 (Sec. III-D)
through the sum over the 2k+1 frequencies of Eq. (18).  Layouts (the project's): samples and bins
are ring-major, (B, L^2); ring k starts at k^2; bin j (|j| <= k) of ring k sits at k^2 + k + j.

ring_dft   bins_k[j] = (1/N_k) sum_n s_k[n] exp(-2 pi i j n / N_k)
ring_idft  s_k[n]    = sum_{|j| <= k} bins_k[j] exp(+2 pi i j n / N_k)

The 1/N_k makes bin j the sum over the orders m = j (mod N_k) of the ring's G_m(theta_k) / 2 pi
(the alias relation behind Eqs. (15) and (18)).  Both are O(N_k^2) sums, with the angle reduced
exactly as (j n mod N_k) / N_k before the cosine and sine are taken.
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _kernel(k, sign):
    """exp(sign 2 pi i j n / N) for j = -k..k (rows) and n = 0..N-1 (columns)."""
    N = 2 * k + 1
    j = np.arange(-k, k + 1, dtype=np.int64)[:, None]
    n = np.arange(N, dtype=np.int64)[None, :]
    ang = TWO_PI * np.mod(j * n, N) / N
    return np.cos(ang) + sign * 1j * np.sin(ang)


def ring_dft(samples, L, rings=None):
    """Bins of every ring by the direct DFT sum.  samples: (B, L^2) or (L^2,) complex.
    ``rings`` (an iterable of k) computes only those rings' bins and leaves the rest zero."""
    s = np.atleast_2d(np.asarray(samples, dtype=np.complex128))
    out = np.zeros_like(s)
    for k in (range(L) if rings is None else sorted(set(rings))):
        N = 2 * k + 1
        ring = s[:, k * k:k * k + N]                         # (B, N)
        out[:, k * k:k * k + N] = (ring @ _kernel(k, -1.0).T) / N
    return out if np.ndim(samples) == 2 else out[0]


def ring_idft(bins, L, rings=None):
    """Samples of every ring from its 2k+1 bins by the direct sum (no scaling); ``rings`` as in
    ring_dft."""
    b = np.atleast_2d(np.asarray(bins, dtype=np.complex128))
    out = np.zeros_like(b)
    for k in (range(L) if rings is None else sorted(set(rings))):
        N = 2 * k + 1
        out[:, k * k:k * k + N] = b[:, k * k:k * k + N] @ _kernel(k, 1.0)
    return out if np.ndim(bins) == 2 else out[0]
