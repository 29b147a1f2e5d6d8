"""Structured O(n^2) per-order solve (Sec. IV-C's complexity discussion), a study kept as a CPU
test: the library's plans keep explicit inverses, and this checks the O(n^2) alternative.

P_m[k][j] = P~_{m+j}^m(theta_k) satisfies the three-term recursion of Sec. III-G along j, so
diag(cos theta) P_m - P_m T = u e_{n-1}^T with T the symmetric tridiagonal recursion (Jacobi) matrix:
displacement rank one.  With T = S diag(lambda) S^T, C = P_m S is Cauchy-like,
C[k][i] = u_k v_i / (x_k - lambda_i) (v = S^T e_{n-1}), and P_m f = g is solved in O(n^2) by
Gaussian elimination with partial pivoting on the generators (u, v) of C (Gohberg, Kailath and
Olshevsky, Math. Comp. 64, 1995), then f = S y; one step of iterative refinement with the residual
g - P_m f brings the error to the float64 level.  The tests pin the displacement identity and the
solve against numpy's LU on the oracle's P~ at the greedy rings.
"""
import numpy as np
import pytest

from oracle import legendre, sampling


def _jacobi(L, m):
    """T (n x n): x P~_{m+j} = P~_{m+j+1} / a_{m+j} + b_{m+j} P~_{m+j-1} (Sec. III-G's recursion)."""
    n = L - m
    T = np.zeros((n, n))
    for j in range(n - 1):
        l = m + j
        off = np.sqrt(((l + 1) ** 2 - m * m) / (4.0 * (l + 1) ** 2 - 1.0))   # 1 / a_l = b_{l+1}
        T[j + 1, j] = off
        T[j, j + 1] = off
    return T


def _cauchy_like_solve(x, u, lam, v, g):
    """C y = g for C[k][i] = u_k v_i / (x_k - lam_i), elimination with partial pivoting on the
    rank-one generators, then the two triangular solves."""
    n = x.size
    x, u, v, g = x.copy(), u.copy(), v.copy(), g.copy()
    Lf, Uf = np.zeros((n, n)), np.zeros((n, n))
    for s in range(n):
        c = u[s:] * v[s] / (x[s:] - lam[s])
        p = s + int(np.argmax(np.abs(c)))
        if p != s:
            for arr in (x, u, g):
                arr[[s, p]] = arr[[p, s]]
            Lf[[s, p], :s] = Lf[[p, s], :s]
            c[[0, p - s]] = c[[p - s, 0]]
        d = c[0]
        r = u[s] * v[s:] / (x[s] - lam[s:])
        Lf[s:, s] = c / d
        Uf[s, s:] = r
        u[s + 1:] -= (c[1:] / d) * u[s]
        v[s + 1:] -= v[s] * (r[1:] / d)
    y = np.zeros_like(g)
    for s in range(n):
        y[s] = g[s] - Lf[s, :s] @ y[:s]
    z = np.zeros_like(g)
    for s in range(n - 1, -1, -1):
        z[s] = (y[s] - Uf[s, s + 1:] @ z[s + 1:]) / Uf[s, s]
    return z


def _setup(L, m):
    th = sampling.thetas(L)
    P = legendre.ptilde_order(m, L, th)[m:, :]      # rings m.. of the ordering, degrees m..L-1
    x = np.cos(th[m:])
    T = _jacobi(L, m)
    R = x[:, None] * P - P @ T
    lam, S = np.linalg.eigh(T)
    return P, x, R, lam, S


@pytest.mark.parametrize("L,m", [(16, 0), (64, 0), (64, 7), (128, 30), (128, 120)])
def test_displacement_rank_one(L, m):
    P, x, R, lam, S = _setup(L, m)
    n = L - m
    # every column but the last vanishes: the recursion closes inside P_m
    assert np.abs(R[:, : n - 1]).max() <= 1e-13 * max(1.0, np.abs(P).max())
    # and the last column is the next degree, P~_L^m(theta_k) / a_{L-1}
    assert np.abs(R[:, n - 1]).max() > 0.0


@pytest.mark.parametrize("L,m", [(64, 0), (64, 5), (128, 0), (128, 60)])
def test_structured_solve_matches_lu(L, m):
    P, x, R, lam, S = _setup(L, m)
    n = L - m
    u, v = R[:, n - 1], S[n - 1, :]
    f = np.random.default_rng(L + m).standard_normal((n, 4))
    g = P @ f
    f0 = S @ _cauchy_like_solve(x, u, lam, v, g)
    f1 = f0 + S @ _cauchy_like_solve(x, u, lam, v, g - P @ f0)       # one refinement step
    f_lu = np.linalg.solve(P, g)
    assert np.abs(f0 - f).max() <= 1e-11
    assert np.abs(f1 - f).max() <= max(1e-13, 2.0 * np.abs(f_lu - f).max())
