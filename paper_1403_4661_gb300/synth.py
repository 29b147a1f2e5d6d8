"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module holds none of the transform's arithmetic: it only turns a seed into numbers.
Generator: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) evaluated counter-style, output i = mix(seed + (i+1) * 0x9E3779B97F4A7C15) mod 2^64;
53-bit uniforms u = (z >> 11) * 2^-53 in [0, 1); normals by Box-Muller from consecutive pairs.

Workload recipes (the paper's experiments draw re/im iid uniform on [-1, 1], Sec. IV-A):
  uniform_coeffs    f_l^m re/im iid U[-1, 1]
  decaying_coeffs   f_l^m re/im iid N(0, 1) * (l + 1)^-1
  uniform_samples   samples re/im iid U[-1, 1]
  normal_samples    real samples iid N(0, 1)
Layouts: coefficients (B, L^2) with f_l^m at l^2 + l + m; samples (B, L^2) ring-major.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, start=0):
    """Outputs start..start+count-1 of the splitmix64 stream for ``seed``, as uint64."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed, count, start=0):
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed, count, start=0):
    return 2.0 * uniform01(seed, count, start) - 1.0


def normal(seed, count, start=0):
    u = uniform01(seed, 2 * count, 2 * start).reshape(count, 2)
    r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    return r * np.cos(2.0 * np.pi * u[:, 1])


def degree_of_index(L):
    """l for every coefficient index l^2 + l + m."""
    return np.repeat(np.arange(L), 2 * np.arange(L) + 1)


def uniform_coeffs(L, batch, seed):
    v = uniform_pm1(seed, 2 * batch * L * L).reshape(batch, L * L, 2)
    return v[..., 0] + 1j * v[..., 1]


def decaying_coeffs(L, batch, seed):
    v = normal(seed, 2 * batch * L * L).reshape(batch, L * L, 2)
    scale = 1.0 / (degree_of_index(L) + 1.0)
    return (v[..., 0] + 1j * v[..., 1]) * scale[None, :]


def uniform_samples(L, batch, seed):
    v = uniform_pm1(seed, 2 * batch * L * L).reshape(batch, L * L, 2)
    return v[..., 0] + 1j * v[..., 1]


def normal_samples(L, batch, seed):
    return normal(seed, batch * L * L).reshape(batch, L * L)


def normal_coeffs(L, batch, seed):
    v = normal(seed, 2 * batch * L * L).reshape(batch, L * L, 2)
    return v[..., 0] + 1j * v[..., 1]


def loguniform_bandlimits(count, lo, hi, seed):
    """L_i = round(exp(U[ln lo, ln hi])) - the uneven-batch recipe."""
    u = uniform01(seed, count)
    return np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)
