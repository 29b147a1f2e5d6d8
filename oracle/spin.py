"""Spin-s spherical harmonic transforms on the optimal-dimensionality sampling, plain float64.

Test infrastructure (oracle); see the package docstring.

Sec. III-H: the forward and inverse transforms carry over to band-limited spin-s functions with
f -> sf, f_l^m -> sf_l^m, Y_l^m -> sY_l^m.  Appendix A defines, for |s| <= l, |m| <= l,
    sY_l^m(theta, phi) = (-1)^s sqrt((2l+1)/(4 pi)) e^{i m phi} d^l_{m,-s}(theta),
with d^l the Wigner small-d function.  The convention of d (rotation e^{-i beta J_y}, matrix element
<l m'| . |l m>) is fixed by the explicit sum
    d^j_{a,b}(beta) = sqrt((j+a)!(j-a)!(j+b)!(j-b)!) sum_t (-1)^(a-b+t)
                      cos(beta/2)^(2j+b-a-2t) sin(beta/2)^(a-b+2t) / ((j+b-t)! t! (a-b+t)! (j-a-t)!),
which gives 1Y_1^0 = sqrt(3/(8 pi)) sin(theta) and reduces to Y_l^m for s = 0 (both checked in
tests/test_oracle_spin.py).

Evaluation, as Appendix A prescribes: a three-term recursion in increasing l at fixed (m, s),
    l sqrt(((l+1)^2 - a^2)((l+1)^2 - b^2)) d^{l+1} = (2l+1)(l(l+1) cos(theta) - a b) d^l
                                                    - (l+1) sqrt((l^2 - a^2)(l^2 - b^2)) d^{l-1},
a = m, b = -s, started at l0 = max(|m|, |s|), where the explicit sum has a single term:
    d^{l0}_{a,b} = (-1)^(a-b+t) sqrt(C) cos(theta/2)^p sin(theta/2)^q,
C an integer ratio of factorials (computed exactly here), p, q the powers of that term.  The start
value underflows float64 for large l0 near the poles, so it is carried as mantissa * 2**exponent
and the recursion rescales like oracle/legendre.py.

Reading of the paper (garbled here, as for the spin-0 recursion): the printed start value has the
powers of cos(theta/2) and sin(theta/2) exchanged relative to the definition (for s = m = 1 the
definition gives -sqrt(3/(4 pi)) sin^2(theta/2), the printed form cos^2(theta/2)) and lacks
sqrt((2m+1)/(4 pi)); the printed recursion matches the one above up to the garbled factor on its
left side.  The definition governs.

Transforms: a spin-s signal has coefficients sf_l^m for |s| <= l < L (L^2 - s^2 of them), stored
in the spin-0 layout (index l^2 + l + m; entries with l < |s| are ignored on input and zero on
output).  The per-order matrices sP_m[k][l] = sP~_l^m(theta_k), rings k >= |m|, degrees
l >= max(|m|, |s|), are square for |m| >= |s| and have more rows than columns for |m| < |s|; there
the solve of Eq. (14) is a least-squares solve, exact for band-limited spin signals.  There is
no P_{-m} = (-1)^m P_m symmetry for s != 0 (sY_l^{-m} relates to (-s)Y_l^m), so every order has
its own table.
"""
import math

import numpy as np

from .sampling import sample_ring_index

TWO_PI = 2.0 * math.pi
RESCALE_BITS = 600
_FLUSH_EXP = -1022


def _frexp_int(n):
    """Non-negative Python integer -> (mantissa in [0.5, 1), exponent), exactly rounded."""
    if n == 0:
        return 0.0, 0
    e = n.bit_length()
    shift = e - 64
    top = n >> shift if shift > 0 else n << (-shift)
    return math.ldexp(float(top), -64), e


def base_term(j, a, b):
    """(sign, C, p, q) of the single term of the explicit sum at j = max(|a|, |b|):
    d^j_{a,b}(beta) = sign sqrt(C) cos(beta/2)^p sin(beta/2)^q."""
    if j != max(abs(a), abs(b)):
        raise ValueError("the start value is taken at j = max(|a|, |b|)")
    t = max(0, b - a)
    assert t == min(j + b, j - a)
    f = math.factorial
    num = f(j + a) * f(j - a) * f(j + b) * f(j - b)
    den = (f(j + b - t) * f(t) * f(a - b + t) * f(j - a - t)) ** 2
    assert num % den == 0
    sign = -1.0 if (a - b + t) % 2 else 1.0
    return sign, num // den, 2 * j + b - a - 2 * t, a - b + 2 * t


def _power_ext(x, n):
    """x**n (x >= 0 array, n >= 0 integer) as (mantissa, exponent) arrays, by n multiplications
    renormalised with frexp after each."""
    v, e = np.frexp(np.ones_like(x))
    for _ in range(n):
        v, de = np.frexp(v * x)
        e = np.where(v == 0.0, 0, e + de)
    return v, e


def base_value(j, a, b, theta):
    """d^j_{a,b}(theta_k) at j = max(|a|, |b|) as (mantissa, exponent) arrays."""
    sign, C, p, q = base_term(j, a, b)
    theta = np.asarray(theta, dtype=np.float64)
    mc, ec = _power_ext(np.cos(theta / 2.0), p)
    ms, es = _power_ext(np.sin(theta / 2.0), q)
    cm, ce = _frexp_int(C)
    if ce % 2:                          # sqrt(cm 2^ce) with an even exponent
        cm, ce = cm * 2.0, ce - 1
    v, de = np.frexp(sign * math.sqrt(cm) * mc * ms)
    e = np.where(v == 0.0, 0, ec + es + de + ce // 2)
    return v, e


def spin_ptilde(s, m, L, theta):
    """sP~_l^m(theta_k) = sY_l^m(theta_k, 0) for l = l0..L-1, l0 = max(|m|, |s|); any integer m.
    Returns an array (K, L - l0) (empty when l0 >= L)."""
    theta = np.asarray(theta, dtype=np.float64)
    a, b = m, -s
    l0 = max(abs(m), abs(s))
    n = L - l0
    out = np.zeros((theta.size, max(n, 0)))
    if n <= 0:
        return out
    x = np.cos(theta)
    sgn = -1.0 if s % 2 else 1.0

    def emit(l, p, e):
        v = np.ldexp(sgn * math.sqrt((2.0 * l + 1.0) / (4.0 * math.pi)) * p, e)
        v[np.abs(v) < 2.0 ** _FLUSH_EXP] = 0.0
        out[:, l - l0] = v

    p, e = base_value(l0, a, b, theta)
    p_prev = np.zeros_like(p)
    emit(l0, p, e)
    for l in range(l0, L - 1):
        if l == 0:                      # a = b = 0: d^1_{00} = cos(theta) d^0_{00}
            nxt = x * p
        else:
            c1 = (2.0 * l + 1.0) * (l * (l + 1.0) * x - a * b)
            c2 = (l + 1.0) * math.sqrt((l * l - a * a) * (l * l - b * b))
            c0 = l * math.sqrt(((l + 1.0) ** 2 - a * a) * ((l + 1.0) ** 2 - b * b))
            nxt = (c1 * p - c2 * p_prev) / c0
        p_prev, p = p, nxt
        big = (np.abs(p) > 2.0 ** RESCALE_BITS) & (e < 0)
        if np.any(big):
            p = np.where(big, np.ldexp(p, -RESCALE_BITS), p)
            p_prev = np.where(big, np.ldexp(p_prev, -RESCALE_BITS), p_prev)
            e = np.where(big, e + RESCALE_BITS, e)
        emit(l + 1, p, e)
    return out


def wigner_d_sum(j, a, b, beta):
    """d^j_{a,b}(beta) by the full explicit sum (every term), for checks at small j."""
    f = math.factorial
    beta = np.asarray(beta, dtype=np.float64)
    pre = math.sqrt(f(j + a) * f(j - a) * f(j + b) * f(j - b))
    out = np.zeros_like(beta)
    for t in range(max(0, b - a), min(j + b, j - a) + 1):
        den = f(j + b - t) * f(t) * f(a - b + t) * f(j - a - t)
        out += ((-1.0) ** (a - b + t) * pre / den * np.cos(beta / 2.0) ** (2 * j + b - a - 2 * t)
                * np.sin(beta / 2.0) ** (a - b + 2 * t))
    return out


def spin_harmonic(s, l, m, theta, phi):
    """sY_l^m(theta, phi) by the definition and the explicit sum (small l only)."""
    return ((-1.0) ** s * math.sqrt((2 * l + 1) / (4 * math.pi)) * wigner_d_sum(l, m, -s, theta)
            * np.exp(1j * m * np.asarray(phi)))


def _coeff_index(l, m):
    return l * l + l + m


def _orders(L):
    return [0] + [v for mm in range(1, L) for v in (mm, -mm)]


def inverse(coeffs, L, theta, s):
    """Samples from spin-s coefficients by Procedure 2 (Sec. III-D with Y -> sY, Sec. III-H):
    G_m(theta_k) = 2 pi sum_l sf_l^m sP~_l^m(theta_k), then f(theta_k, phi_n) = (1/2 pi)
    sum_m e^{i m phi_n} G_m(theta_k) at every sample."""
    c = np.atleast_2d(np.asarray(coeffs, dtype=np.complex128))
    theta = np.asarray(theta, dtype=np.float64)
    k_idx, n_idx, N = sample_ring_index(L)
    f = np.zeros((c.shape[0], L * L), dtype=np.complex128)
    for m in _orders(L):
        l0 = max(abs(m), abs(s))
        if l0 >= L:
            continue
        P = spin_ptilde(s, m, L, theta)                        # (L rings, L - l0)
        G = TWO_PI * (c[:, _coeff_index(np.arange(l0, L), m)] @ P.T)
        ang = TWO_PI * np.mod(m * n_idx, N) / N
        f += (np.cos(ang) + 1j * np.sin(ang))[None, :] * G[:, k_idx] / TWO_PI
    return f if np.ndim(coeffs) == 2 else f[0]


def forward(samples, L, theta, s):
    """Spin-s coefficients from samples by Procedure 1 (Sec. III-C with Y -> sY, Sec. III-H), in
    the spatial domain: for |m| = L-1..0 and both signs, g_m[k] = (2 pi/N_k) sum_n f(theta_k,
    phi_n) e^{-i m phi_n} on the rings k >= |m|, solve 2 pi sP_m f_m = g_m (least squares when
    |m| < |s|), then subtract f~_m (Eq. (16) with sY) from the samples of the rings k < |m|."""
    x = np.atleast_2d(np.asarray(samples, dtype=np.complex128))
    theta = np.asarray(theta, dtype=np.float64)
    f = x.copy()
    out = np.zeros_like(f)
    k_idx, n_idx, N = sample_ring_index(L)
    ring_start = np.arange(L, dtype=np.int64) ** 2
    for mm in range(L - 1, -1, -1):
        j0 = mm * mm
        seg = ring_start[mm:] - j0
        Nk = 2.0 * np.arange(mm, L) + 1.0
        solved = []
        for m in ([mm, -mm] if mm > 0 else [0]):
            l0 = max(abs(m), abs(s))
            if l0 >= L:
                continue
            P = spin_ptilde(s, m, L, theta)                    # all rings, l = l0..L-1
            ang = TWO_PI * np.mod(m * n_idx[j0:], N[j0:]) / N[j0:]
            ph = np.cos(ang) + 1j * np.sin(ang)
            g = TWO_PI / Nk * np.add.reduceat(f[:, j0:] * np.conj(ph)[None, :], seg, axis=1)
            A = TWO_PI * P[mm:, :]
            if A.shape[0] == A.shape[1]:
                fm = np.linalg.solve(A, g.T).T
            else:
                fm = np.linalg.lstsq(A, g.T, rcond=None)[0].T
            out[:, _coeff_index(np.arange(l0, L), m)] = fm
            solved.append((m, P, fm))
        if mm > 0:
            for m, P, fm in solved:                            # rings k < |m|: f <- f - f~_m
                G = TWO_PI * (fm @ P[:mm, :].T)
                ang = TWO_PI * np.mod(m * n_idx[:j0], N[:j0]) / N[:j0]
                f[:, :j0] -= (np.cos(ang) + 1j * np.sin(ang))[None, :] * G[:, k_idx[:j0]] / TWO_PI
    return out if np.ndim(samples) == 2 else out[0]


def dense_matrix(L, theta, s):
    """Brute force A[(k,n),(l,m)] = sY_l^m(theta_k, phi_kn) by the explicit sum, l >= |s|;
    columns of l < |s| are zero.  Small L only."""
    k_idx, n_idx, N = sample_ring_index(L)
    th = np.asarray(theta, dtype=np.float64)[k_idx]
    ph = TWO_PI * n_idx / N
    A = np.zeros((L * L, L * L), dtype=np.complex128)
    for l in range(abs(s), L):
        for m in range(-l, l + 1):
            A[:, _coeff_index(l, m)] = spin_harmonic(s, l, m, th, ph)
    return A


def dense_forward(samples, A, s):
    """Least-squares solve over the columns l >= |s| (the others stay 0)."""
    L2 = A.shape[1]
    L = int(round(math.sqrt(L2)))
    cols = np.arange(s * s, L2)
    x = np.atleast_2d(samples)
    out = np.zeros((x.shape[0], L2), dtype=np.complex128)
    out[:, cols] = np.linalg.lstsq(A[:, cols], x.T, rcond=None)[0].T
    return out
