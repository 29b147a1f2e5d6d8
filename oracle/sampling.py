"""Sampling layout and ring ordering, plain float64.

Test infrastructure (oracle); see the package docstring.

Sec. III-A: L iso-latitude rings; ring k (the k-th entry of the ordered vector theta, Eq. (7))
carries 2k+1 equispaced longitudes phi = 2 pi n / (2k+1), n = 0..2k (Eq. (8)), so the scheme has
sum_k (2k+1) = L^2 samples (Eq. (9)).  Samples are stored ring-major: ring k at offset k^2.

Sec. III-E: rings sit on the equiangular set Theta_t = pi (2t+1)/(2L-1), t = 0..L-1 (Eq. (19)).
Two orderings of Theta into theta are given:
  * the simple ordering of Eq. (20): theta_0 = pi, then alternately from the north and the south
    towards the equator, ending at pi (2 floor((L-1)/2) + 1)/(2L-1);
  * the condition-number-minimisation ordering: theta_{L-1} is fixed to the ring farthest from the
    poles; for m = L-2, ..., 0, theta_m is the unused element of Theta that minimises the condition
    number of P_m (Eq. (12)) built from theta_m..theta_{L-1}.
Reading: "condition number" is the 2-norm one, sigma_max / sigma_min (the paper's wording "ratio of
the largest eigenvalue to the smallest" is not defined for a non-symmetric P_m); exact ties go to
the lowest index t.

Sec. III-F (alternative placement): the sets Theta^1 and Theta^2 put the L rings at equal steps of
the measures sin(theta) d theta and |tan(theta)|^(1/3) d theta, starting from Theta_0 = pi (the
south pole): the measure between consecutive elements is 1/L of its integral over [0, pi]
(2/L and 2 pi/(L sqrt 3)).  Here they are built literally from that definition (numerical
integration, root finding) and sorted ascending like Eq. (19), so that the same index orderings
(Eq. (20) or condition-number minimisation) turn them into theta^1, theta^2.  The ring kept
farthest from the poles is the element nearest pi/2 (for Eq. (19) that is index floor((L-1)/2)).
"""
import math

import numpy as np

from .legendre import ptilde_order, sectoral_bases


def ring_offsets(L):
    """Offset of ring k in a ring-major sample vector: k^2 (Eq. (9))."""
    return np.arange(L, dtype=np.int64) ** 2


def sample_ring_index(L):
    """For every sample j: (ring k, longitude index n, ring length N = 2k+1)."""
    k = np.repeat(np.arange(L, dtype=np.int64), 2 * np.arange(L) + 1)
    n = np.arange(L * L, dtype=np.int64) - k * k
    return k, n, 2 * k + 1


def sample_phi(L):
    """phi of every sample, Eq. (8): 2 pi n / (2k+1)."""
    k, n, N = sample_ring_index(L)
    return 2.0 * math.pi * n / N


def equiangular_set(L):
    """Theta_t = pi (2t+1)/(2L-1), t = 0..L-1 (Eq. (19))."""
    t = np.arange(L, dtype=np.float64)
    return math.pi * (2.0 * t + 1.0) / (2.0 * L - 1.0)


def _cumulative_measure(measure):
    """C(x) = measure of [x, pi] for the placement measures of Sec. III-F."""
    from scipy import integrate

    if measure == "sin":
        return lambda x: integrate.quad(math.sin, x, math.pi, epsabs=1e-13, epsrel=1e-13)[0]
    if measure != "tan13":
        raise ValueError(measure)
    # F(x) = integral of |tan t|^(1/3) over [0, x].  For x <= pi/2 the substitutions u = tan t,
    # w = u^(1/3) turn it into the integral of 3 w^3 / (1 + w^6) over [0, W], W = tan(x)^(1/3); the
    # part beyond w = 1, with v = 1/w, is the integral of 3 v / (1 + v^6) over [1/W, 1].  Both
    # integrands are smooth on [0, 1].  |tan| is symmetric about pi/2: F(x) = 2 F(pi/2) - F(pi - x).
    f = lambda w: 3.0 * w ** 3 / (1.0 + w ** 6)   # noqa: E731
    f_inv = lambda v: 3.0 * v / (1.0 + v ** 6)    # noqa: E731
    q = lambda fn, a, b: integrate.quad(fn, a, b, epsabs=1e-14, epsrel=1e-13)[0]   # noqa: E731
    half = q(f, 0.0, 1.0) + q(f_inv, 0.0, 1.0)

    def F_left(x):
        W = math.tan(x) ** (1.0 / 3.0) if x < math.pi / 2 else np.inf
        if W <= 1.0:
            return q(f, 0.0, W)
        return half - q(f_inv, 0.0, 1.0 / W)

    def F(x):
        return F_left(x) if x <= math.pi / 2 else 2.0 * half - F_left(math.pi - x)

    return lambda x: 2.0 * half - F(x)


def measure_set(L, measure="uniform"):
    """The ring set of a placement rule, ascending: "uniform" is Eq. (19); "sin" and "tan13" are
    Theta^1 and Theta^2 of Sec. III-F: Theta_0 = pi and, for t = 1..L-1, the measure of
    [Theta_t, Theta_{t-1}] equal to 1/L of the measure of [0, pi], i.e. C(Theta_t) = t C(0) / L
    with C(x) the measure of [x, pi]."""
    if measure == "uniform":
        return equiangular_set(L)
    from scipy import optimize

    C = _cumulative_measure(measure)
    step = C(0.0) / L
    out = [math.pi]
    for t in range(1, L):
        out.append(optimize.brentq(lambda x: C(x) - t * step, 0.0, out[-1], xtol=1e-15, rtol=1e-15))
    return np.sort(np.array(out))


def middle_index(Theta):
    """Index of the element of Theta nearest pi/2; mirror pairs (equal distance up to rounding,
    within 1e-12) go to the lowest index."""
    d = np.abs(np.asarray(Theta) - math.pi / 2)
    return int(np.nonzero(d <= d.min() + 1e-12)[0][0])


# Reading for the mirror-symmetric sets Theta^1, Theta^2: reflecting a ring about pi/2 multiplies
# its row of P_m by (-1)^(l+m) column by column, an orthogonal change that leaves the condition
# number unchanged whenever the fixed rows are themselves symmetric, so mirror candidates tie
# exactly in exact arithmetic and rounding would break the tie arbitrarily.  For those sets the
# greedy takes the lowest index among candidates within a relative 1e-9 of the smallest condition
# number.  Eq. (19) has no mirror pairs (pi - Theta_t is never in it); its rule stays exact ties.
TIE_RTOL = {"uniform": 0.0, "sin": 1e-9, "tan13": 1e-9}


def _pick(cand, kappa, rtol):
    kappa = np.asarray(kappa, dtype=np.float64)
    if rtol == 0.0:
        return cand[int(np.argmin(kappa))]
    kmin = kappa.min()
    return cand[int(np.nonzero(kappa <= kmin * (1.0 + rtol))[0][0])] if np.isfinite(kmin) else cand[0]


def simple_order(L):
    """Indices t into Theta for the ordering of Eq. (20): [L-1, 0, L-2, 1, L-3, 2, ...]."""
    order = [L - 1]
    lo, hi = 0, L - 2
    take_lo = True
    while len(order) < L:
        if take_lo:
            order.append(lo)
            lo += 1
        else:
            order.append(hi)
            hi -= 1
        take_lo = not take_lo
    return np.array(order, dtype=np.int64)


def _order_block(m, L, theta_vals):
    """P~_l^m at the given co-latitudes, l = m..L-1 (rows follow theta_vals)."""
    return ptilde_order(m, L, theta_vals)


def cond_exact(P):
    """2-norm condition number by a full SVD (reading of Sec. III-E)."""
    s = np.linalg.svd(P, compute_uv=False)
    if s[-1] == 0.0:
        return np.inf
    return s[0] / s[-1]


def greedy_order_exact(L, measure="uniform"):
    """Condition-number-minimisation ordering (Sec. III-E), every candidate scored by a full SVD,
    on the ring set of `measure` (measure_set).

    Returns the indices t into the set for theta_0..theta_{L-1}.  O(L^5); meant for L <= ~64.
    """
    Theta = measure_set(L, measure)
    order = np.full(L, -1, dtype=np.int64)
    order[L - 1] = (L - 1) // 2 if measure == "uniform" else middle_index(Theta)
    used = {order[L - 1]}
    for m in range(L - 2, -1, -1):
        # the full table P~_l^m(Theta_t), l = m..L-1, for every t
        T = _order_block(m, L, Theta)
        fixed = T[order[m + 1:]]
        cand = np.array([t for t in range(L) if t not in used], dtype=np.int64)
        kappa = [cond_exact(np.vstack([T[t][None, :], fixed])) for t in cand]
        best_t = _pick(cand, kappa, TIE_RTOL[measure])   # all singular: the lowest unused index
        order[m] = best_t
        used.add(best_t)
    return order


def _bisect_secular(mu, z2, lo, hi, iters=200):
    """Root of 1 + sum_i z2_i / (mu_i - x) = 0 on (lo, hi), vectorised over rows of z2.

    f is increasing on the bracket; plain bisection to float64 resolution.
    """
    lo = np.array(lo, dtype=np.float64)
    hi = np.array(hi, dtype=np.float64)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.all((mid == lo) | (mid == hi)):
            break
        with np.errstate(divide="ignore", invalid="ignore"):
            f = 1.0 + np.sum(z2 / (mu[None, :] - mid[:, None]), axis=1)
        neg = ~(f >= 0.0)  # f < 0 (or nan at a pole): the root lies above mid
        lo = np.where(neg, mid, lo)
        hi = np.where(neg, hi, mid)
    return 0.5 * (lo + hi)


def greedy_order_secular(L, measure="uniform"):
    """Same ordering as ``greedy_order_exact``, with each candidate scored through the rank-one
    update of the fixed block's Gram matrix (O(L^4) overall).

    For order m let B be the fixed (n-1) x n block (rows theta_{m+1..L-1}, columns l = m..L-1) and
    r a candidate row.  P_m^T P_m = B^T B + r r^T; with B^T B = V diag(mu) V^T (mu ascending) and
    z = V^T r, the eigenvalues of P_m^T P_m are the roots of 1 + sum_i z_i^2/(mu_i - x) = 0; by
    interlacing the smallest lies in [mu_0, mu_1] and the largest in [mu_max, mu_max + |r|^2].
    kappa = sqrt(largest / smallest).
    """
    Theta = measure_set(L, measure)
    order = np.full(L, -1, dtype=np.int64)
    order[L - 1] = (L - 1) // 2 if measure == "uniform" else middle_index(Theta)
    used = np.zeros(L, dtype=bool)
    used[order[L - 1]] = True
    bases = sectoral_bases(L, Theta)
    for m in range(L - 2, -1, -1):
        T = ptilde_order(m, L, Theta, bases)
        fixed = T[order[m + 1:]]
        cand = np.nonzero(~used)[0]
        R = T[cand]
        if cand.size == 1:
            order[m] = cand[0]
            used[cand[0]] = True
            continue
        mu, V = np.linalg.eigh(fixed.T @ fixed)
        mu = np.maximum(mu, 0.0)
        Z2 = (R @ V) ** 2
        r2 = np.sum(R * R, axis=1)
        n = mu.size
        if n == 1:
            lam_min = r2  # 1x1 system: P_m = [r]
            lam_max = r2
        else:
            lam_min = _bisect_secular(mu, Z2, np.full(cand.size, mu[0]), np.full(cand.size, mu[1]))
            lam_max = _bisect_secular(mu, Z2, np.full(cand.size, mu[-1]), mu[-1] + r2)
        with np.errstate(divide="ignore", invalid="ignore"):
            kappa = np.where(lam_min > 0.0, np.sqrt(lam_max / lam_min), np.inf)
        pick = _pick(cand, kappa, TIE_RTOL[measure])
        order[m] = pick
        used[pick] = True
    return order


def thetas(L, ordering="greedy", measure="uniform"):
    """The ordered co-latitude vector theta (Eq. (7)) for an ordering rule, on the ring set of a
    placement measure (Eq. (19) by default; Theta^1, Theta^2 of Sec. III-F)."""
    Theta = measure_set(L, measure)
    if ordering == "simple":
        return Theta[simple_order(L)]
    if ordering == "greedy":
        return Theta[greedy_order_secular(L, measure)]
    if ordering == "greedy_exact":
        return Theta[greedy_order_exact(L, measure)]
    raise ValueError(ordering)


def order_conditions(L, theta):
    """kappa(P_m) for m = 0..L-1 (2-norm, full SVD) - the planner diagnostic of Figs. 3-4."""
    bases = sectoral_bases(L, theta)
    out = np.zeros(L)
    for m in range(L):
        P = ptilde_order(m, L, theta[m:], (bases[0][:, m:], bases[1][:, m:]))
        out[m] = cond_exact(P)
    return out
