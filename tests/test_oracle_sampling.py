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
