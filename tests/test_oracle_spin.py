"""Pins of the spin-s oracle (oracle/spin.py; Sec. III-H, Appendix A).

External references: sympy's Wigner small-d (an independent implementation, same rotation
convention as the definition), the textbook spin-weighted harmonics 1Y_1^m, 2Y_2^0, 2Y_2^2.
Invariants: the unitarity sum rule sum_m |sY_l^m|^2 = (2l+1)/(4 pi), orthonormality over the sphere
(Gauss-Legendre nodes in cos(theta) x equispaced phi, exact for these polynomial integrands), the
conjugation rule conj(sY_l^m) = (-1)^(s+m) (-s)Y_l^(-m), and the reduction to Y_l^m at s = 0.
Transforms: the dense brute force of sY at the sample points (inverse = A c, forward = least squares).
"""
import math

import numpy as np
import pytest

from oracle import legendre, sampling, spin
from paper_1403_4661_gb300 import synth

TH = np.array([1e-3, 0.2, 0.9, math.pi / 2, 2.1, 3.0, math.pi - 1e-3])


def test_textbook_spin_harmonics():
    th = TH
    # values at phi = 0 of 1Y_1^0 = sqrt(3/8pi) sin, 1Y_1^1 = -sqrt(3/16pi)(1 - cos) e^{i phi},
    # 1Y_1^-1 = -sqrt(3/16pi)(1 + cos) e^{-i phi}, 2Y_2^0 = sqrt(15/32pi) sin^2,
    # 2Y_2^2 = sqrt(5/64pi)(1 - cos)^2 e^{2 i phi}, (-1)Y_1^0 = -sqrt(3/8pi) sin
    cases = [(1, 0, 1, math.sqrt(3 / (8 * math.pi)) * np.sin(th)),
             (1, 1, 1, -math.sqrt(3 / (16 * math.pi)) * (1 - np.cos(th))),
             (1, -1, 1, -math.sqrt(3 / (16 * math.pi)) * (1 + np.cos(th))),
             (2, 0, 2, math.sqrt(15 / (32 * math.pi)) * np.sin(th) ** 2),
             (2, 2, 2, math.sqrt(5 / (64 * math.pi)) * (1 - np.cos(th)) ** 2),
             (-1, 0, 1, -math.sqrt(3 / (8 * math.pi)) * np.sin(th))]
    for s, m, l, ref in cases:
        P = spin.spin_ptilde(s, m, l + 1, th)
        l0 = max(abs(m), abs(s))
        np.testing.assert_allclose(P[:, l - l0], ref, atol=1e-15)


def test_against_sympy_wigner_d():
    import sympy
    from sympy.physics.quantum.spin import Rotation

    def d(l, a, b, t):
        v = complex(sympy.N(Rotation.d(l, a, b, float(t)).doit()))
        assert abs(v.imag) < 1e-12   # the small-d function is real
        return v.real

    th = np.array([0.3, 1.7, 2.9])
    L = 7
    for s in (-2, -1, 1, 2, 3):
        for m in range(-(L - 1), L):
            l0 = max(abs(m), abs(s))
            if l0 >= L:
                continue
            P = spin.spin_ptilde(s, m, L, th)
            for l in range(l0, L):
                ref = np.array([(-1) ** s * math.sqrt((2 * l + 1) / (4 * math.pi)) *
                                d(l, m, -s, t) for t in th])
                np.testing.assert_allclose(P[:, l - l0], ref, atol=1e-14, err_msg=f"s={s} m={m} l={l}")


def test_spin_zero_is_the_scalar_basis():
    L = 300
    th = np.concatenate([TH, sampling.equiangular_set(40)])
    bases = legendre.sectoral_bases(L, th)
    for m in (0, 1, 7, 150, 299, -3, -298):
        a = spin.spin_ptilde(0, m, L, th)
        b = legendre.ptilde_signed(m, L, th, bases)
        np.testing.assert_allclose(a, b, rtol=0, atol=2e-12 * np.abs(b).max())


@pytest.mark.parametrize("s", [1, 2, -2])
def test_unitarity_sum_rule_including_underflow_range(s):
    # sum over all orders m of |sY_l^m(theta)|^2 = (2l+1)/(4 pi) at every theta, up to l = 400,
    # which exercises the extended-exponent start values near the poles; the recursion loses
    # ~l^2 u relative next to the poles (as the scalar one does), hence 1e-11
    L = 401
    th = np.array([0.01, 0.5, 1.3, 2.6, math.pi - 0.02])
    acc = np.zeros((th.size, L))
    for m in range(-(L - 1), L):
        l0 = max(abs(m), abs(s))
        if l0 >= L:
            continue
        acc[:, l0:] += spin.spin_ptilde(s, m, L, th) ** 2
    l = np.arange(L)
    want = (2 * l + 1) / (4 * math.pi)
    np.testing.assert_allclose(acc[:, abs(s):], np.broadcast_to(want[abs(s):], acc[:, abs(s):].shape), rtol=1e-11)


def test_orthonormality_on_the_sphere():
    s, L = 2, 20
    x, w = np.polynomial.legendre.leggauss(2 * L + 4)
    th = np.arccos(x)
    nphi = 2 * L + 3
    phi = 2 * math.pi * np.arange(nphi) / nphi
    rows = []
    for m in range(-(L - 1), L):
        l0 = max(abs(m), abs(s))
        if l0 >= L:
            continue
        P = spin.spin_ptilde(s, m, L, th)
        for l in range(l0, L):
            rows.append(np.outer(P[:, l - l0], np.exp(1j * m * phi)).ravel())
    Y = np.array(rows)
    wq = np.repeat(w, nphi) * (2 * math.pi / nphi)
    G = (Y * wq[None, :]) @ Y.conj().T
    np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-13)


def test_conjugation_rule():
    L = 30
    for s in (1, 2):
        for m in range(-(L - 1), L):
            if max(abs(m), s) >= L:
                continue
            a = spin.spin_ptilde(s, m, L, TH)
            b = spin.spin_ptilde(-s, -m, L, TH)
            np.testing.assert_allclose(a, (-1.0) ** (s + m) * b, atol=1e-14)


@pytest.mark.parametrize("s", [1, 2, -1])
def test_transforms_against_dense_brute_force(s):
    L = 7
    th = sampling.thetas(L, "greedy")
    A = spin.dense_matrix(L, th, s)
    c = synth.uniform_coeffs(L, 2, 21)
    c[:, : s * s] = 0.0
    x = spin.inverse(c, L, th, s)
    np.testing.assert_allclose(x, c @ A.T, atol=1e-13)
    # the dense least squares recovers c; Procedure 1 agrees with it to its own error level
    np.testing.assert_allclose(spin.dense_forward(x, A, s), c, atol=1e-13)
    got = spin.forward(x, L, th, s)
    assert np.abs(got - c).max() < 1e-9


def test_planted_mistake_printed_start_value_is_caught():
    # the start value as printed (powers of cos(theta/2), sin(theta/2) exchanged) fails the
    # textbook value 1Y_1^1 = -sqrt(3/16pi)(1 - cos theta)
    th = TH
    printed = -math.sqrt(3 / (4 * math.pi)) * np.cos(th / 2) ** 2
    ref = -math.sqrt(3 / (16 * math.pi)) * (1 - np.cos(th))
    assert np.abs(printed - ref).max() > 0.1
    np.testing.assert_allclose(spin.spin_ptilde(1, 1, 2, th)[:, 0], ref, atol=1e-15)
