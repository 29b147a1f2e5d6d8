"""Pins of the oracle's forward (Procedure 1) and inverse (Procedure 2) transforms.

Brute force: the dense L^2 x L^2 system of scipy's Y_l^m at the sampling points (inverse = A c,
forward = A^{-1} s).  Special inputs: Y_00, single modes compared with scipy's Y_l^m at the
sample points.  Invariants: the two round trips of Sec. IV-A (Exps. 1 and 2; the second closes
because any L^2 samples are band-limited in this scheme), linearity, the symmetry of real signals
(f_l^{-m} = (-1)^m conj f_l^m, from Eq. (30)), and the adjoint identities.
"""
import math

import numpy as np
import pytest

from oracle import sampling, sht
from paper_1403_4661_gb300 import synth


def _theta(L, ordering="greedy"):
    return sampling.thetas(L, ordering)


@pytest.mark.parametrize("L", [1, 2, 3, 6, 11, 16])
def test_against_dense_brute_force(L):
    th = _theta(L)
    A = sht.dense_matrix(L, th)
    c = synth.uniform_coeffs(L, 2, 11)
    s = synth.uniform_samples(L, 2, 12)
    np.testing.assert_allclose(sht.inverse(c, L, th), sht.dense_inverse(c, A), atol=1e-13 * L)
    np.testing.assert_allclose(sht.forward(s, L, th), sht.dense_forward(s, A), atol=1e-12)
    np.testing.assert_allclose(sht.inverse_adjoint(s, L, th), sht.dense_inverse_adjoint(s, A), atol=1e-13 * L)


def test_dense_brute_force_simple_ordering():
    L = 10
    th = _theta(L, "simple")
    A = sht.dense_matrix(L, th)
    s = synth.uniform_samples(L, 1, 3)
    np.testing.assert_allclose(sht.forward(s, L, th), sht.dense_forward(s, A), atol=1e-11)


def test_y00():
    L = 9
    th = _theta(L)
    c = np.zeros(L * L, dtype=np.complex128)
    c[0] = 1.0
    s = sht.inverse(c, L, th)
    np.testing.assert_allclose(s, np.full(L * L, 1.0 / math.sqrt(4 * math.pi)), atol=1e-15)
    np.testing.assert_allclose(sht.forward(s, L, th), c, atol=1e-14)


def test_single_modes_match_scipy():
    from scipy.special import sph_harm_y

    L = 10
    th = _theta(L)
    k, n, N = sampling.sample_ring_index(L)
    phi = 2 * math.pi * n / N
    eye = np.eye(L * L, dtype=np.complex128)
    S = sht.inverse(eye, L, th)                  # row i = samples of basis function i
    C = sht.forward(S, L, th)
    for l in range(L):
        for m in range(-l, l + 1):
            i = l * l + l + m
            np.testing.assert_allclose(S[i], sph_harm_y(l, m, th[k], phi), atol=1e-13)
    np.testing.assert_allclose(C, eye, atol=1e-12)


@pytest.mark.parametrize("L", [32, 64])
def test_round_trips_exp1_exp2(L):
    th = _theta(L)
    c = synth.uniform_coeffs(L, 3, 21)
    e1 = sht.errors_spectral(c, sht.forward(sht.inverse(c, L, th), L, th))
    s = synth.uniform_samples(L, 3, 22)
    e2 = sht.errors_spatial(s, sht.inverse(sht.forward(s, L, th), L, th))
    assert e1[0] < 1e-12 and e2[0] < 1e-12


def test_linearity_and_real_symmetry():
    L = 20
    th = _theta(L)
    x = synth.normal_samples(L, 2, 5)            # real signals
    c = sht.forward(x, L, th)
    for l in range(L):
        for m in range(1, l + 1):
            np.testing.assert_allclose(c[:, l * l + l - m], (-1) ** m * np.conj(c[:, l * l + l + m]), atol=1e-13)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    y = synth.uniform_samples(L, 2, 6)
    np.testing.assert_allclose(sht.forward(a * x + b * y, L, th),
                               a * sht.forward(x, L, th) + b * sht.forward(y, L, th), atol=1e-12)


def test_adjoint_dot_products():
    L = 40
    th = _theta(L)
    c = synth.normal_coeffs(L, 1, 1)[0]
    y = synth.uniform_samples(L, 1, 2)[0]
    lhs = np.vdot(y, sht.inverse(c, L, th))
    rhs = np.vdot(sht.inverse_adjoint(y, L, th), c)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_dense_forward_adjoint_consistency():
    L = 8
    th = _theta(L)
    A = sht.dense_matrix(L, th)
    w = synth.normal_coeffs(L, 1, 3)[0]
    s = synth.uniform_samples(L, 1, 4)[0]
    z = sht.dense_forward_adjoint(w, A)[0]
    # <F s, w> = <s, F^H w>
    assert abs(np.vdot(w, sht.forward(s, L, th)) - np.vdot(z, s)) < 1e-12


def test_evaluate_samples_matches_inverse():
    L = 30
    th = _theta(L)
    c = synth.decaying_coeffs(L, 2, 8)
    idx = np.array([0, 1, 7, 100, 401, L * L - 1])
    np.testing.assert_allclose(sht.evaluate_samples(c, L, th, idx), sht.inverse(c, L, th)[:, idx], atol=1e-13)


@pytest.mark.parametrize("L", [1, 5, 17, 40])
def test_evaluate_at_arbitrary_points_matches_scipy(L):
    """Eq. (6) at random (theta, phi), not on the sampling grid: the oracle's evaluate against the
    plain sum of scipy's Y_l^m (Condon-Shortley phase, orthonormal, Eq. (29))."""
    from scipy.special import sph_harm_y

    rng = np.random.default_rng(L)
    th = np.concatenate([[0.0, math.pi, 1e-3, math.pi / 2], rng.uniform(0, math.pi, 12)])
    ph = np.concatenate([[0.3, 2.0, 6.0, 0.0], rng.uniform(0, 2 * math.pi, 12)])
    c = synth.uniform_coeffs(L, 2, 40 + L)
    ref = np.zeros((2, th.size), dtype=np.complex128)
    for l in range(L):
        for m in range(-l, l + 1):
            ref += c[:, l * l + l + m][:, None] * sph_harm_y(l, m, th, ph)[None, :]
    got = sht.evaluate(c, L, th, ph)
    np.testing.assert_allclose(got, ref, atol=1e-12 * max(1, L))


# --- planted mistakes: each plausible error in the oracle must fail a pin above -------------

def test_planted_mistakes_are_caught(monkeypatch):
    from oracle import legendre

    L = 6
    th = _theta(L)
    A = sht.dense_matrix(L, th)
    c = synth.uniform_coeffs(L, 1, 1)
    good = sht.dense_inverse(c, A)
    orig = legendre.ptilde_order

    def no_cs_phase(m, L_, theta, bases=None):      # Condon-Shortley phase dropped
        return orig(m, L_, theta, bases) * (-1.0) ** m

    def wrong_normalisation(m, L_, theta, bases=None):
        return orig(m, L_, theta, bases) * (1.0 + 1e-3 * m)

    for bad in (no_cs_phase, wrong_normalisation):
        monkeypatch.setattr(sht, "ptilde_order", bad)
        assert np.abs(sht.inverse(c, L, th) - good).max() > 1e-6
        monkeypatch.setattr(sht, "ptilde_order", orig)
