"""Pins of the oracle's sampling layout and ring orderings (Sec. III-A, III-E).

The equiangular set and the simple ordering are checked against the values the paper prints
(Eqs. (19), (20)); the fast greedy planner against the exact-SVD greedy; the greedy's structure
against what the paper states (theta_{L-1} farthest from the poles) and what follows from it
(the pole ring, singular for every m >= 1, is left for m = 0).  The condition numbers are
regression values of this code (the paper's Figs. 3-4 are plots without printed values).
"""
import math
import os

import numpy as np
import pytest

from oracle import sampling

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_sample_count_and_layout():
    for L in [1, 2, 5, 16]:
        k, n, N = sampling.sample_ring_index(L)
        assert k.size == L * L                             # Eq. (9)
        assert np.all(N == 2 * k + 1)
        assert np.all((n >= 0) & (n < N))
        np.testing.assert_array_equal(sampling.ring_offsets(L), np.arange(L) ** 2)
    phi = sampling.sample_phi(3)
    np.testing.assert_allclose(phi[4:9], 2 * math.pi * np.arange(5) / 5)   # Eq. (8), ring k = 2


def test_equiangular_and_simple_order_match_eqs_19_20():
    L = 12
    T = sampling.equiangular_set(L)
    np.testing.assert_allclose(T, math.pi * (2 * np.arange(L) + 1) / (2 * L - 1))
    th = T[sampling.simple_order(L)]
    printed = [math.pi, math.pi / (2 * L - 1), math.pi * (2 * L - 3) / (2 * L - 1), 3 * math.pi / (2 * L - 1)]
    np.testing.assert_allclose(th[:4], printed)
    np.testing.assert_allclose(th[-1], math.pi * (2 * ((L - 1) // 2) + 1) / (2 * L - 1))
    for L in [1, 2, 7, 12, 33]:
        assert sorted(sampling.simple_order(L)) == list(range(L))


@pytest.mark.parametrize("L", [2, 3, 8, 16, 24, 32])
def test_greedy_fast_equals_exact(L):
    np.testing.assert_array_equal(sampling.greedy_order_secular(L), sampling.greedy_order_exact(L))


@pytest.mark.parametrize("L", [16, 32, 48])
def test_greedy_structure(L):
    o = sampling.greedy_order_secular(L)
    assert sorted(o) == list(range(L))
    assert o[L - 1] == (L - 1) // 2          # farthest from the poles
    assert o[0] == L - 1                     # Theta_{L-1} = pi: singular P_m for every m >= 1


def test_condition_numbers_regression():
    # survey-time and oracle agree; values of this code, not printed in the paper
    expect_greedy = {16: 5.1604, 32: 7.6112, 48: 8.8972}
    expect_simple = {16: 5.1604, 32: 39.357, 48: 603.22}
    for L in expect_greedy:
        T = sampling.equiangular_set(L)
        kg = sampling.order_conditions(L, T[sampling.greedy_order_secular(L)]).max()
        ks = sampling.order_conditions(L, T[sampling.simple_order(L)]).max()
        assert abs(kg - expect_greedy[L]) < 1e-3 * expect_greedy[L]
        assert abs(ks - expect_simple[L]) < 1e-3 * expect_simple[L]


def test_golden_orders_are_permutations():
    for L in [512, 1024]:
        path = os.path.join(GOLDEN, f"ring_order_L{L}.txt")
        if not os.path.exists(path):
            pytest.skip("golden ordering not generated")
        o = np.loadtxt(path, dtype=np.int64, comments="#")
        assert sorted(o.tolist()) == list(range(L))
        assert o[L - 1] == (L - 1) // 2 and o[0] == L - 1


def _tan13_integral(x):
    """Integral of |tan t|^(1/3) over [0, x], x in [0, pi], in closed form (an independent method
    from the oracle's numerical integration): with T = tan(x)^(2/3) and t = tan^(2/3), the
    integrand becomes (3/2) T / (1 + T^3) dT, whose partial fractions -1/(3(1+T)) +
    (T+1)/(3(T^2-T+1)) integrate to h(T) below; |tan| is symmetric about pi/2."""
    half = math.pi / math.sqrt(3.0)

    def left(y):
        if y >= math.pi / 2:
            return half
        T = math.tan(y) ** (2.0 / 3.0)
        h = (-math.log1p(T) / 3.0 + math.log(T * T - T + 1.0) / 6.0
             + (math.atan((2.0 * T - 1.0) / math.sqrt(3.0)) + math.pi / 6.0) / math.sqrt(3.0))
        return 1.5 * h

    return left(x) if x <= math.pi / 2 else 2.0 * half - left(math.pi - x)


@pytest.mark.parametrize("L", [8, 17, 32])
def test_alternative_measure_sets_pinned(L):
    """Theta^1 (sin measure) against its closed form cos Theta_t = 2t/L - 1; Theta^2 (|tan|^(1/3)
    measure) against the closed-form integral: the measure of [Theta_t, pi] is t/L of the total
    2 pi/sqrt(3); both start at the south pole and are mirror-symmetric about pi/2 apart from it."""
    T1 = sampling.measure_set(L, "sin")
    np.testing.assert_allclose(T1, np.sort(np.arccos(2.0 * np.arange(L) / L - 1.0)), atol=1e-13, rtol=0)
    T2 = sampling.measure_set(L, "tan13")
    total = 2.0 * math.pi / math.sqrt(3.0)
    for t, x in enumerate(T2[::-1]):          # Theta_0 = pi first
        if t == 0:
            continue   # Theta_0 = pi by definition (asserted below); the measure is flat there
        # the angle whose closed-form measure of [angle, pi] is t/L of the total, by bisection
        # (compared as angles: next to pi/2 the measure changes steeply with the angle)
        lo, hi = 0.0, math.pi
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if total - _tan13_integral(mid) > total * t / L:
                lo = mid
            else:
                hi = mid
        assert abs(x - 0.5 * (lo + hi)) < 1e-13, t
    for T in (T1, T2):
        assert T[-1] == math.pi
        u = T[:-1]
        np.testing.assert_allclose(u + u[::-1], math.pi, atol=1e-13, rtol=0)
    np.testing.assert_array_equal(sampling.measure_set(L, "uniform"), sampling.equiangular_set(L))


@pytest.mark.parametrize("L", [6, 9, 12, 16])
@pytest.mark.parametrize("measure", ["sin", "tan13"])
def test_greedy_fast_equals_exact_on_alternative_sets(L, measure):
    np.testing.assert_array_equal(sampling.greedy_order_secular(L, measure),
                                  sampling.greedy_order_exact(L, measure))


def test_kappa_study_of_alternative_measures():
    """Sec. III-F: rings placed by the measures sin(theta) d theta and |tan(theta)|^(1/3) d theta
    make the P_m far worse conditioned than the equiangular set, and condition-number minimisation
    does not rescue them (the paper shows this in figures only; the values are this code's)."""
    L = 32
    k = {(ms, od): sampling.order_conditions(L, sampling.thetas(L, od, ms)).max()
         for ms in ("uniform", "sin", "tan13") for od in ("simple", "greedy")}
    expect = {("uniform", "simple"): 39.3565, ("uniform", "greedy"): 7.61121,
              ("sin", "simple"): 2.64023e9, ("sin", "greedy"): 2.64023e9,
              ("tan13", "simple"): 3.78515e11, ("tan13", "greedy"): 3.78515e11}
    for key, v in expect.items():
        assert abs(k[key] - v) <= 1e-3 * v, (key, k[key])
    for ms in ("sin", "tan13"):
        assert k[ms, "greedy"] > 1e8 * k["uniform", "greedy"]
        assert k[ms, "greedy"] > 0.5 * k[ms, "simple"]      # reordering does not help
    assert k["uniform", "greedy"] < k["uniform", "simple"] / 5  # it does for Eq. (19)
