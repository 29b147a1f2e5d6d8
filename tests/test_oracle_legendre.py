"""Pins of the oracle's P~_l^m(theta) = Y_l^m(theta, 0) against things other than itself.

Definition: Sec. III-B and Appendix A, Eq. (29) (orthonormal, Condon-Shortley phase); symmetry
Eq. (23).  Pins: closed forms for l <= 2 typed from the textbook expressions, scipy's
sph_harm_y, mpmath's arbitrary-precision spherical harmonics (extended exponent range),
Unsold's theorem sum_m |Y_l^m|^2 = (2l+1)/(4 pi), the pole values, and orthonormality by
Gauss-Legendre quadrature.
"""
import math

import numpy as np
import pytest

from oracle.legendre import ptilde_order, ptilde_signed, sectoral_bases

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

RNG = np.random.default_rng(7)
THETA = np.concatenate([RNG.uniform(0.0, math.pi, 40), [1e-3, 0.5, math.pi / 2, math.pi - 1e-3]])


def test_closed_forms_l_le_2():
    L = 3
    x, s = np.cos(THETA), np.sin(THETA)
    q = 1.0 / math.sqrt(math.pi)
    expect = {
        (0, 0): np.full_like(THETA, 0.5 * q),
        (1, 0): 0.5 * math.sqrt(3.0) * q * x,
        (1, 1): -0.5 * math.sqrt(1.5) * q * s,
        (2, 0): 0.25 * math.sqrt(5.0) * q * (3 * x * x - 1),
        (2, 1): -0.5 * math.sqrt(7.5) * q * s * x,
        (2, 2): 0.25 * math.sqrt(7.5) * q * s * s,
    }
    for (l, m), v in expect.items():
        got = ptilde_order(m, L, THETA)[:, l - m]
        np.testing.assert_allclose(got, v, rtol=1e-14, atol=1e-15)
        # negative orders, Eq. (23)
        gotn = ptilde_signed(-m, L, THETA)[:, l - m]
        np.testing.assert_allclose(gotn, (-1) ** m * v, rtol=1e-14, atol=1e-15)


def test_matches_scipy_up_to_l100():
    from scipy.special import sph_harm_y

    L = 101
    bases = sectoral_bases(L, THETA)
    for m in [0, 1, 2, 7, 30, 64, 100]:
        got = ptilde_order(m, L, THETA, bases)
        for l in range(m, L, 3):
            ref = sph_harm_y(l, m, THETA, 0.0).real
            np.testing.assert_allclose(got[:, l - m], ref, rtol=1e-10, atol=1e-13)
        # negative orders through Eq. (23), against scipy's own Y_l^{-m} (not the symmetry)
        gotn = ptilde_signed(-m, L, THETA, bases)
        for l in range(m, L, 7):
            ref = sph_harm_y(l, -m, THETA, 0.0).real
            np.testing.assert_allclose(gotn[:, l - m], ref, rtol=1e-10, atol=1e-13)


def test_extended_range_against_mpmath():
    """Large m near the poles: the sectoral start underflows float64, the result does not."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    L = 2048
    cases = [(1500, 0.55), (1800, 0.75), (1000, 0.2), (2000, 1.3), (1200, 0.45)]
    th = np.array([t for _, t in cases])
    bases = sectoral_bases(L, th)
    for i, (m, t) in enumerate(cases):
        got = ptilde_order(m, L, th[i:i + 1], (bases[0][:, i:i + 1], bases[1][:, i:i + 1]))[0]
        for l in [m, m + 1, m + 17, (m + L) // 2, L - 1]:
            ref = float(mpmath.re(mpmath.spherharm(l, m, mpmath.mpf(t), 0)))
            if abs(ref) < 1e-300:
                assert abs(got[l - m]) < 1e-290
            else:
                assert abs(got[l - m] - ref) <= 1e-12 * max(abs(ref), 1e-300) + 1e-300, (m, t, l)


def test_unsold_sum():
    L = 512
    th = np.array([1e-4, 0.01, 0.3, 1.0, math.pi / 2, 2.5, math.pi - 1e-4])
    bases = sectoral_bases(L, th)
    tot = np.zeros((th.size, L))
    for m in range(L):
        P = ptilde_order(m, L, th, bases)
        w = 1.0 if m == 0 else 2.0  # +-m, Eq. (23)
        tot[:, m:] += w * P * P
    ell = np.arange(L)
    # the forward recursion loses ~l^2 u relative accuracy next to the poles (Sec. III-G's method
    # itself, measured against mpmath: 2.4e-11 at l = 1023, theta = pi/2047); any wrong term would
    # be off by O(1)
    np.testing.assert_allclose(tot, np.broadcast_to((2 * ell + 1) / (4 * math.pi), tot.shape),
                               rtol=2e-11)


def test_pole_values():
    L = 200
    th = np.array([0.0, math.pi])
    bases = sectoral_bases(L, th)
    ell = np.arange(L)
    P0 = ptilde_order(0, L, th, bases)
    np.testing.assert_allclose(P0[0], np.sqrt((2 * ell + 1) / (4 * math.pi)), rtol=1e-13)
    np.testing.assert_allclose(P0[1], (-1.0) ** ell * np.sqrt((2 * ell + 1) / (4 * math.pi)), rtol=1e-13)
    # sin(pi) is 1.2e-16 in float64, so m >= 1 vanishes to that order only
    for m in [1, 2, 50, 199]:
        assert np.all(np.abs(ptilde_order(m, L, th, bases)) < 1e-13)


@pytest.mark.parametrize("L", [16, 64, 200])
def test_orthonormal_by_gauss_legendre(L):
    x, w = np.polynomial.legendre.leggauss(L)
    th = np.arccos(x)
    bases = sectoral_bases(L, th)
    for m in sorted({0, 1, L // 3, L // 2, L - 2, L - 1}):
        P = ptilde_order(m, L, th, bases)
        gram = 2.0 * math.pi * (P.T * w) @ P
        np.testing.assert_allclose(gram, np.eye(L - m), atol=1e-12)
