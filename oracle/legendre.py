"""Scaled associated Legendre functions P~_l^m(theta) = Y_l^m(theta, 0), plain float64.

Test infrastructure (oracle); see the package docstring.

Definition (Sec. III-B, text after Eq. (11); Appendix A, Eq. (29)):
    P~_l^m(theta) = N_l^m P_l^m(cos theta),  N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
with the Condon-Shortley phase (-1)^m inside P_l^m, and for negative order (Eq. (23)):
    P~_l^{-m} = (-1)^m P~_l^m.

Evaluation (Sec. III-G): three-term recursion in increasing degree l at fixed order m, started from
the sectoral value P~_m^m, with adaptive rescaling so that the start value, which underflows float64
for large m near the poles, is carried as mantissa * 2**exponent.

Reading of the paper (it is garbled here): the recursion and base condition as printed
(Eqs. (21), (22)) do not satisfy the definition P~ = Y_l^m(theta, 0) (the printed recursion fails
already at (l, m) = (1, 0) and the printed base lacks sqrt((2m+1)/(4 pi))).  The definition governs,
so this module uses the recursion that follows from it:
    P~_0^0       = 1 / sqrt(4 pi)
    P~_m^m       = -sqrt((2m+1)/(2m)) sin(theta) P~_{m-1}^{m-1}
    P~_{m+1}^m   = sqrt(2m+3) cos(theta) P~_m^m
    P~_l^m       = a_lm (cos(theta) P~_{l-1}^m - b_lm P~_{l-2}^m),
        a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)),  b_lm = sqrt(((l-1)^2 - m^2) / (4 (l-1)^2 - 1)).
Values whose magnitude falls below 2**-1022 are returned as 0 (their contribution to any sum in
the transforms is below 1e-300).
"""
import math

import numpy as np

# A mantissa that grows past 2**RESCALE_BITS is divided by 2**RESCALE_BITS and the exponent raised.
RESCALE_BITS = 600
_FLUSH_EXP = -1022


def sectoral_bases(L, theta):
    """Return (mant, expo) with P~_m^m(theta_k) = mant[m, k] * 2**expo[m, k] for m = 0..L-1.

    Product recursion P~_m^m = -sqrt((2m+1)/(2m)) sin(theta) P~_{m-1}^{m-1} (derived from the
    definition, Appendix A), renormalised with frexp after every step so nothing underflows.
    """
    theta = np.asarray(theta, dtype=np.float64)
    s = np.sin(theta)
    mant = np.zeros((L, theta.size))
    expo = np.zeros((L, theta.size), dtype=np.int64)
    v, e = np.frexp(np.full(theta.size, 1.0 / math.sqrt(4.0 * math.pi)))
    mant[0], expo[0] = v, e
    for m in range(1, L):
        v = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * v
        v, de = np.frexp(v)
        e = e + de
        e = np.where(v == 0.0, 0, e)
        mant[m], expo[m] = v, e
    return mant, expo


def ptilde_order(m, L, theta, bases=None):
    """P~_l^m(theta_k) for one order m >= 0, all k, l = m..L-1.  Returns array (K, L - m).

    Sec. III-G: recursion in increasing l at fixed m, with adaptive rescaling of the start value.
    """
    if m < 0:
        raise ValueError("ptilde_order takes m >= 0; use P~^{-m} = (-1)^m P~^m (Eq. (23))")
    theta = np.asarray(theta, dtype=np.float64)
    if bases is None:
        bases = sectoral_bases(m + 1, theta)
    mant, expo = bases[0][m].copy(), bases[1][m].copy()
    x = np.cos(theta)
    n = L - m
    out = np.zeros((theta.size, n))

    def emit(col, p, e):
        # value = p * 2**e, flushed to 0 below 2**-1022
        v = np.ldexp(p, e)
        v[np.abs(v) < 2.0 ** _FLUSH_EXP] = 0.0
        out[:, col] = v

    p_prev = np.zeros_like(mant)
    p = mant
    e = expo
    emit(0, p, e)
    if n == 1:
        return out
    p_prev, p = p, math.sqrt(2.0 * m + 3.0) * x * p
    emit(1, p, e)
    for l in range(m + 2, L):
        a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
        b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
        p_prev, p = p, a * (x * p - b * p_prev)
        big = (np.abs(p) > 2.0 ** RESCALE_BITS) & (e < 0)
        if np.any(big):
            p = np.where(big, np.ldexp(p, -RESCALE_BITS), p)
            p_prev = np.where(big, np.ldexp(p_prev, -RESCALE_BITS), p_prev)
            e = np.where(big, e + RESCALE_BITS, e)
        emit(l - m, p, e)
    return out


def ptilde_signed(m, L, theta, bases=None):
    """P~_l^m(theta_k) for any order |m| < L, l = |m|..L-1, using Eq. (23) for m < 0."""
    block = ptilde_order(abs(m), L, theta, bases)
    if m < 0 and (abs(m) % 2 == 1):
        block = -block
    return block
