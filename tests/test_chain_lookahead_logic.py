"""The forward chain's blocked look-ahead (the tensor-core chain kernel's block structure), restated
on the host with random tables and checked against the plain order-by-order chain of Eqs.
(14)-(16).  Both run in float64 numpy; the test pins the index logic the kernel relies on:

* row j of g_m (ring m + j, bins +-m) is reached only by the orders m + 2j + 1 and above, so in a
  block [lo, hi] of kB orders every row j >= J_m = floor((hi - m + 1)/2) is final at the block's
  start and only the leading "tracked" rows wait for orders of the same block;
* the alias contribution of order m' at ring k is Q_m'[k] g_m' with Q_m' = P~_m' P_m'^{-1}, so the
  tracked rows follow from the final rows (X1) and a recurrence over the block's orders (X2);
* the block's solves (Y), alias products (Z) and the subtraction from the rings below the block
  (E, skipping the block's own rows) then reproduce the sequential chain.

Layouts as in the library: order-major bins, block m at rows_off(L, m), row k - m, four columns
per signal (bin +m re/im, bin -m re/im; bin 0 in the first pair only).
"""
import numpy as np
import pytest

KB = 32


def alias_bin(m, k):
    N = 2 * k + 1
    return (m + k) % N - k


def rows_off(L, m):
    return m * L - m * (m - 1) // 2


def blk_J(i):
    return (i + 1) >> 1


def blk_offH(i):
    p = i >> 1
    return p * p + (i & 1) * p


def alias_map(a, g):
    """Where order m's (G+, G-) land in the four columns of row (|a|, ring k)."""
    if a == 0:
        return np.array([g[0] + g[2], g[1] + g[3], 0.0, 0.0])
    if a > 0:
        return g.copy()
    return np.array([g[2], g[3], g[0], g[1]])


def _tables(L, B, seed):
    rng = np.random.default_rng(seed)
    W0 = rng.standard_normal((rows_off(L, L), 4 * B))
    W0[0:L, 2::4] = 0.0   # order 0: bin 0 only
    W0[0:L, 3::4] = 0.0
    Pt = [rng.standard_normal((L, L - m)) for m in range(L)]
    Pi = [rng.standard_normal((L - m, L - m)) / np.sqrt(L - m) for m in range(L)]
    return W0, Pt, Pi


def _sequential(L, B, W0, Pt, Pi):
    W, F = W0.copy(), {}
    for m in range(L - 1, -1, -1):
        n = L - m
        F[m] = Pi[m] @ W[rows_off(L, m):rows_off(L, m) + n]
        for k in range(m):
            G = Pt[m][k] @ F[m]
            a = alias_bin(m, k)
            o = abs(a)
            for s in range(B):
                W[rows_off(L, o) + k - o, 4 * s:4 * s + 4] -= alias_map(a, G[4 * s:4 * s + 4])
    return F


def _blocked(L, B, W0, Pt, Pi):
    W, F = W0.copy(), {}
    Q = {}
    for m in range(L):
        hi = L - 1 - ((L - 1 - m) // KB) * KB
        lo = max(0, hi - KB + 1)
        Q[m] = Pt[m][lo:m] @ Pi[m]
    hi = L - 1
    while hi >= 0:
        lo = max(0, hi - KB + 1)
        nb = hi - lo + 1
        nE = blk_offH(nb)
        # X1: contributions through the final rows, per (order, ring) pair
        X1 = {}
        for ip in range(nb):
            mp = hi - ip
            for kk in range(mp - lo):
                k = lo + kk
                a = alias_bin(mp, k)
                o = abs(a)
                if o < lo or k - o >= blk_J(hi - o):
                    continue
                Jp = blk_J(ip)
                X1[(ip, kk)] = Q[mp][kk][Jp:] @ W[rows_off(L, mp) + Jp:rows_off(L, mp) + L - mp]
        # X2: tracked entries, then the recurrence over the block's orders, per signal
        for s in range(B):
            hs = np.zeros((nE, 4))
            for e in range(nE):
                i = 0
                while blk_offH(i + 1) <= e:
                    i += 1
                m, j = hi - i, e - blk_offH(i)
                k = m + j
                v = W[rows_off(L, m) + j, 4 * s:4 * s + 4].copy()
                for mp in range(hi, k, -1):
                    a = alias_bin(mp, k)
                    if abs(a) == m:
                        v -= alias_map(a, X1[(hi - mp, k - lo)][4 * s:4 * s + 4])
                hs[e] = v
            for ip in range(nb):
                mp, Jp = hi - ip, blk_J(ip)
                if Jp == 0:
                    continue
                h = hs[blk_offH(ip):blk_offH(ip) + Jp].copy()
                for kk in range(mp - lo):
                    k = lo + kk
                    a = alias_bin(mp, k)
                    o = abs(a)
                    if o < lo or k - o >= blk_J(hi - o):
                        continue
                    hs[blk_offH(hi - o) + (k - o)] -= alias_map(a, Q[mp][kk][:Jp] @ h)
            for e in range(nE):
                i = 0
                while blk_offH(i + 1) <= e:
                    i += 1
                W[rows_off(L, hi - i) + e - blk_offH(i), 4 * s:4 * s + 4] = hs[e]
        # Y: every order's solve from its now final g_m
        for i in range(nb):
            m = hi - i
            F[m] = Pi[m] @ W[rows_off(L, m):rows_off(L, m) + L - m]
        if lo == 0:
            break
        # Z, E: alias products, subtracted from the rows that later blocks read
        G = {i: Pt[hi - i][:hi - i] @ F[hi - i] for i in range(nb) if hi - i > 0}
        for k in range(hi):
            for mp in range(hi, max(lo, k + 1) - 1, -1):
                a = alias_bin(mp, k)
                o = abs(a)
                if o >= lo:
                    continue
                for s in range(B):
                    W[rows_off(L, o) + k - o, 4 * s:4 * s + 4] -= alias_map(a, G[hi - mp][k, 4 * s:4 * s + 4])
        hi -= KB
    return F


def test_block_geometry():
    # J(i) rows for the order hi - i; offH is their prefix sum; 256 tracked rows per full block
    assert [blk_J(i) for i in range(6)] == [0, 1, 1, 2, 2, 3]
    for n in range(1, 40):
        assert blk_offH(n) == sum(blk_J(i) for i in range(n))
    assert blk_offH(KB) == 256


def test_rows_reached_only_from_m_plus_2j_plus_1():
    # every order m' > ring k that lands in bin +-m of ring k = m + j satisfies m' >= m + 2j + 1
    for k in range(1, 60):
        for mp in range(k + 1, 200):
            m = abs(alias_bin(mp, k))
            assert mp >= m + 2 * (k - m) + 1


@pytest.mark.parametrize("L,B", [(1, 1), (2, 1), (5, 2), (31, 1), (32, 2), (33, 1), (40, 2), (70, 1)])
def test_blocked_chain_reproduces_sequential_chain(L, B):
    W0, Pt, Pi = _tables(L, B, L)
    Fs = _sequential(L, B, W0, Pt, Pi)
    Fb = _blocked(L, B, W0, Pt, Pi)
    for m in range(L):
        scale = max(1.0, float(np.abs(Fs[m]).max()))
        assert np.abs(Fb[m] - Fs[m]).max() <= 1e-12 * scale, m
