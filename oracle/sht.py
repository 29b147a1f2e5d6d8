"""Forward and inverse SHT on the optimal-dimensionality sampling, plain float64.

Test infrastructure (oracle); see the package docstring.

Layouts (the paper fixes none; these are the project's):
  samples      (B, L^2) complex, ring-major: ring k at offset k^2, sample n at phi = 2 pi n/(2k+1)
  coefficients (B, L^2) complex, f_l^m at index l^2 + l + m

inverse  - Procedure 2 (Sec. III-D) taken literally: for m = 0..L-1 evaluate P~^{+-m}, form
           G_{+-m}(theta_k) by Eq. (11) and add f~_m of Eq. (16) at every sample (Eq. (18)).
forward  - Procedure 1 (Sec. III-C) taken literally in the spatial domain: for m = L-1..0 form
           g_{+-m} from the rings k >= m by the ring DFT at frequency +-m (Eq. (11)), solve
           Eq. (14) with P_m of Eq. (12) (P_{-m} = (-1)^m P_m, Remark 1), then subtract f~_m
           (Eq. (16)) from every sample of the rings k < m (Eqs. (15), (17)).
dense_*  - brute force: the L^2 x L^2 system A[(k,n),(l,m)] = Y_l^m(theta_k, phi_kn) built from
           scipy's spherical harmonics, for small L only.

Readings: Procedure 1 asks for a "(2m+1)-point FFT along each phi-ring"; ring k has 2k+1 points,
so g_m(theta_k) is taken from ring k's own (2k+1)-point DFT at frequency m, which is exact because
after the updates of the steps m' > k ring k holds only orders |m'| <= k.  Exp. 1 draws
coefficients for 0 < l < L; this code transforms every 0 <= l < L.
"""
import math

import numpy as np

from .legendre import ptilde_order, sectoral_bases
from .sampling import sample_ring_index

TWO_PI = 2.0 * math.pi


def _phase(L, m, j0=0, j1=None, layout=None):
    """exp(i m phi_j) for samples j0..j1-1, with the angle reduced exactly: (m n mod N)/N."""
    k, n, N = sample_ring_index(L) if layout is None else layout
    if j1 is None:
        j1 = L * L
    k, n, N = k[j0:j1], n[j0:j1], N[j0:j1]
    r = np.mod(m * n, N)
    ang = TWO_PI * r / N
    return np.cos(ang) + 1j * np.sin(ang), k


def _coeff_index(l, m):
    return l * l + l + m


def inverse(coeffs, L, theta, m_lo=0, orders=None):
    """Samples from coefficients by Procedure 2.  coeffs: (B, L^2) or (L^2,) complex.

    m_lo > 0 runs only the iterations m >= m_lo of the procedure's loop; ``orders`` (an iterable of
    m) runs only those iterations.  Either gives a bounded sample of the work, used to time the
    oracle at large L; the result is then a partial sum.
    """
    c = np.atleast_2d(np.asarray(coeffs, dtype=np.complex128))
    theta = np.asarray(theta, dtype=np.float64)
    Bn = c.shape[0]
    f = np.zeros((Bn, L * L), dtype=np.complex128)
    bases = sectoral_bases(L, theta)
    layout = sample_ring_index(L)
    for m in (range(m_lo, L) if orders is None else sorted(set(orders))):
        # step 1: P~_l^m(theta_k), P~_l^{-m} = (-1)^m P~_l^m, all k, l = m..L-1
        P = ptilde_order(m, L, theta, bases)            # (L rings, L - m)
        ell = np.arange(m, L)
        # step 2: G_{+-m}(theta_k) = 2 pi sum_l f_l^{+-m} P~_l^{+-m}(theta_k)   (Eq. (11))
        Gp = TWO_PI * (c[:, _coeff_index(ell, m)] @ P.T)
        ph, kj = _phase(L, m, layout=layout)
        # step 3: f~_m = (e^{i m phi} G_m + e^{-i m phi} G_{-m}) / 2 pi         (Eq. (16))
        ft = ph[None, :] * Gp[:, kj]
        if m > 0:
            sgn = -1.0 if (m % 2) else 1.0
            Gm = TWO_PI * sgn * (c[:, _coeff_index(ell, -m)] @ P.T)
            ft = ft + np.conj(ph)[None, :] * Gm[:, kj]
        # step 4: f <- f + f~_m                                                   (Eq. (18))
        f += ft / TWO_PI
    return f if np.ndim(coeffs) == 2 else f[0]


def forward(samples, L, theta, m_lo=0, orders=None):
    """Coefficients from samples by Procedure 1.  samples: (B, L^2) or (L^2,) complex.

    m_lo > 0 stops the procedure's loop after the iteration m = m_lo; ``orders`` (an iterable of
    m) runs only those iterations, in the procedure's order.  Either gives a bounded sample of the
    work, used to time the oracle at large L; coefficients of the skipped orders are then 0 and
    the others are not those of the full procedure.
    """
    s = np.atleast_2d(np.asarray(samples, dtype=np.complex128))
    theta = np.asarray(theta, dtype=np.float64)
    Bn = s.shape[0]
    f = s.copy()
    out = np.zeros((Bn, L * L), dtype=np.complex128)
    bases = sectoral_bases(L, theta)
    layout = sample_ring_index(L)
    ring_start = np.arange(L, dtype=np.int64) ** 2
    for m in (range(L - 1, m_lo - 1, -1) if orders is None else sorted(set(orders), reverse=True)):
        P = ptilde_order(m, L, theta, bases)            # P~_l^m(theta_k), all k, l = m..L-1
        ell = np.arange(m, L)
        # step 3: g_{+-m}[k] = (2 pi / N_k) sum_n f(theta_k, phi_n) e^{-+ i m phi_n}, k = m..L-1
        j0 = m * m
        ph, kj = _phase(L, m, j0, layout=layout)
        seg = ring_start[m:] - j0
        Nk = 2.0 * np.arange(m, L) + 1.0
        gp = TWO_PI / Nk * np.add.reduceat(f[:, j0:] * np.conj(ph)[None, :], seg, axis=1)
        # step 4-5: P_m = 2 pi [P~_l^m(theta_k)]_{k,l >= m}  (Eq. (12)); solve Eq. (14)
        Pm = TWO_PI * P[m:, :]
        fp = np.linalg.solve(Pm, gp.T).T                # (B, L - m)
        out[:, _coeff_index(ell, m)] = fp
        if m > 0:
            gm = TWO_PI / Nk * np.add.reduceat(f[:, j0:] * ph[None, :], seg, axis=1)
            sgn = -1.0 if (m % 2) else 1.0
            fm = np.linalg.solve(sgn * Pm, gm.T).T     # P_{-m} = (-1)^m P_m
            out[:, _coeff_index(ell, -m)] = fm
            # step 6-7: rings k < m (samples j < m^2): f <- f - f~_m              (Eqs. (15)-(17))
            Gp = TWO_PI * (fp @ P[:m, :].T)            # G_m(theta_k), k < m
            Gm = TWO_PI * sgn * (fm @ P[:m, :].T)      # G_{-m}(theta_k), k < m
            phl, kl = _phase(L, m, 0, j0, layout=layout)
            ft = (phl[None, :] * Gp[:, kl] + np.conj(phl)[None, :] * Gm[:, kl]) / TWO_PI
            f[:, :j0] -= ft
    return out if np.ndim(samples) == 2 else out[0]


def evaluate(coeffs, L, theta_pts, phi_pts):
    """f(theta, phi) = sum_{l<L} sum_{|m|<=l} f_l^m Y_l^m(theta, phi) at arbitrary points (Eq. (6)).

    coeffs (B, L^2); theta_pts, phi_pts (K,).  Returns (B, K).  O(L^2 K): used to check sampled
    outputs of full-size transforms one point at a time.
    """
    c = np.atleast_2d(np.asarray(coeffs, dtype=np.complex128))
    th = np.asarray(theta_pts, dtype=np.float64)
    ph = np.asarray(phi_pts, dtype=np.float64)
    bases = sectoral_bases(L, th)
    out = np.zeros((c.shape[0], th.size), dtype=np.complex128)
    for m in range(L):
        P = ptilde_order(m, L, th, bases)                  # (K, L - m)
        ell = np.arange(m, L)
        out += (c[:, _coeff_index(ell, m)] @ P.T) * np.exp(1j * m * ph)[None, :]
        if m > 0:
            sgn = -1.0 if (m % 2) else 1.0
            out += sgn * (c[:, _coeff_index(ell, -m)] @ P.T) * np.exp(-1j * m * ph)[None, :]
    return out


def evaluate_samples(coeffs, L, theta, idx):
    """The band-limited signal (Eq. (6)) at the sampling points with ring-major indices ``idx``.

    Same sum as ``evaluate``, with the longitude phases reduced exactly, (m n mod N)/N.
    """
    c = np.atleast_2d(np.asarray(coeffs, dtype=np.complex128))
    k_all, n_all, N_all = sample_ring_index(L)
    idx = np.asarray(idx, dtype=np.int64)
    k, n, N = k_all[idx], n_all[idx], N_all[idx]
    th = np.asarray(theta, dtype=np.float64)[k]
    bases = sectoral_bases(L, th)
    out = np.zeros((c.shape[0], idx.size), dtype=np.complex128)
    for m in range(L):
        P = ptilde_order(m, L, th, bases)
        ell = np.arange(m, L)
        ang = TWO_PI * np.mod(m * n, N) / N
        ph = np.cos(ang) + 1j * np.sin(ang)
        out += (c[:, _coeff_index(ell, m)] @ P.T) * ph[None, :]
        if m > 0:
            sgn = -1.0 if (m % 2) else 1.0
            out += sgn * (c[:, _coeff_index(ell, -m)] @ P.T) * np.conj(ph)[None, :]
    return out


# ----------------------------------------------------------------------------------------------
# Adjoints (for the autograd checks).  The inverse is the linear map c -> A c with
# A[(k,n),(l,m)] = P~_l^m(theta_k) e^{i m phi_kn}  (Eqs. (6), (11), (18)); its adjoint is the plain
# conjugate-transpose sum below.  The forward is A^{-1}, whose adjoint A^{-H} has no cheaper plain
# form than a dense solve, so it is given for small L only (dense_forward_adjoint).
# ----------------------------------------------------------------------------------------------

def inverse_adjoint(samples, L, theta):
    """A^H y: (A^H y)_l^m = sum_k P~_l^m(theta_k) sum_n e^{-i m phi_kn} y_kn."""
    y = np.atleast_2d(np.asarray(samples, dtype=np.complex128))
    theta = np.asarray(theta, dtype=np.float64)
    Bn = y.shape[0]
    out = np.zeros((Bn, L * L), dtype=np.complex128)
    bases = sectoral_bases(L, theta)
    layout = sample_ring_index(L)
    ring_start = np.arange(L, dtype=np.int64) ** 2
    for m in range(0, L):
        P = ptilde_order(m, L, theta, bases)
        ell = np.arange(m, L)
        ph, kj = _phase(L, m, layout=layout)
        hp = np.add.reduceat(y * np.conj(ph)[None, :], ring_start, axis=1)   # (B, L rings)
        out[:, _coeff_index(ell, m)] = hp @ P
        if m > 0:
            sgn = -1.0 if (m % 2) else 1.0
            hm = np.add.reduceat(y * ph[None, :], ring_start, axis=1)
            out[:, _coeff_index(ell, -m)] = sgn * (hm @ P)
    return out if np.ndim(samples) == 2 else out[0]


def dense_matrix(L, theta):
    """Brute force A[(k,n),(l,m)] = Y_l^m(theta_k, phi_kn) from scipy's spherical harmonics."""
    from scipy.special import sph_harm_y

    k, n, N = sample_ring_index(L)
    th = np.asarray(theta, dtype=np.float64)[k]
    ph = 2.0 * math.pi * n / N
    A = np.zeros((L * L, L * L), dtype=np.complex128)
    for l in range(L):
        for m in range(-l, l + 1):
            A[:, _coeff_index(l, m)] = sph_harm_y(l, m, th, ph)
    return A


def dense_inverse(coeffs, A):
    return np.atleast_2d(coeffs) @ A.T


def dense_forward(samples, A):
    return np.linalg.solve(A, np.atleast_2d(samples).T).T


def dense_inverse_adjoint(samples, A):
    return np.atleast_2d(samples) @ A.conj()


def dense_forward_adjoint(coeffs, A):
    """(A^{-1})^H w = A^{-H} w, by a dense solve with A^H."""
    return np.linalg.solve(A.conj().T, np.atleast_2d(coeffs).T).T


def errors_spectral(c_true, c_rec):
    """E^1_max, E^1_mean of Eqs. (25), (26)."""
    d = np.abs(np.asarray(c_true) - np.asarray(c_rec))
    return float(d.max()), float(d.mean())


def errors_spatial(s_true, s_rec):
    """E^2_max, E^2_mean of Eqs. (27), (28)."""
    d = np.abs(np.asarray(s_true) - np.asarray(s_rec))
    return float(d.max()), float(d.mean())
