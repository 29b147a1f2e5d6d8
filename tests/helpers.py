"""Shared helpers of the tests: oracle ring orderings (computed, or read from tests/golden)."""
import functools
import math
import os

import numpy as np

from oracle import sampling

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@functools.lru_cache(maxsize=None)
def oracle_order(L):
    path = os.path.join(GOLDEN, f"ring_order_L{L}.txt")
    if os.path.exists(path):
        return np.loadtxt(path, dtype=np.int64, comments="#")
    return sampling.greedy_order_secular(L)


def oracle_thetas(L):
    return math.pi * (2.0 * oracle_order(L) + 1.0) / (2.0 * L - 1.0)


def tol_samples(s):
    """1e-11 relative to the signal's largest sample: an inverse output sums up to 2 L^2 terms of
    size up to |P~| ~ sqrt(2L / 4 pi), and the oracle's own float64 error is of that order."""
    return 1e-11 * max(1.0, float(np.abs(s).max()))
