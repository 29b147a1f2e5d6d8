"""Write sampled oracle outputs at large band-limits, for the GPU parity tests at full size.

Calls only oracle/ (and the seeded input generator paper_1403_4661_gb300/synth.py, which holds no
arithmetic of the method).  For each L given:
  c   = synth.decaying_coeffs(L, 1, SEED)     f_l^m re/im iid N(0,1) / (l+1)  (the workload recipe)
  s   = oracle.sht.inverse(c)                  Procedure 2 (Sec. III-D)
  c_r = oracle.sht.forward(s)                  Procedure 1 (Sec. III-C)
on the rings of the stored oracle ordering tests/golden/ring_order_L{L}.txt (Sec. III-E), and
writes tests/golden/oracle_L{L}.txt: a header (L, seed, recipe, the oracle's own Exp. 1 errors
E1_max = max |c - c_r| and E1_mean (Eqs. (25), (26)), sha256 of the full c_r and s arrays) and the
values of c_r at seeded coefficient indices and of s at seeded sample indices, 17 significant
digits.  The full arrays (64 MB at L = 2048) are too large to store; the samples are what the
GPU tests compare.

    python tests/golden/make_oracle_reference.py 1024 2048
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import sampling  # noqa: E402
from oracle import sht as osht  # noqa: E402
from paper_1403_4661_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SEED = 1000            # signal 0 of the benchmark workload's batch (seed 1000 + rank 0)
N_COEF = {1024: 2048, 2048: 4096}
N_SAMP = {1024: 512, 2048: 1024}


def indices(L, n_coef, n_samp):
    """Seeded index choice: every coefficient of order m = 0 and m = +-1 up to a quarter of the
    budget (the low orders carry the largest error, Sec. IV-A), the rest uniform without
    repetition; sample indices uniform without repetition, plus ring 0 and the last ring's first
    sample."""
    rng = np.random.default_rng(L)
    low = []
    for l in range(L):
        low.append(l * l + l)
        if l >= 1:
            low += [l * l + l + 1, l * l + l - 1]
    low = np.array(low[: n_coef // 4], dtype=np.int64)
    rest = np.setdiff1d(np.arange(L * L), low)
    ci = np.sort(np.concatenate([low, rng.choice(rest, n_coef - low.size, replace=False)]))
    si = np.unique(np.concatenate([[0, (L - 1) ** 2], rng.choice(L * L, n_samp, replace=False)]))
    return ci, si[:n_samp]


def main(L):
    order = np.loadtxt(os.path.join(HERE, f"ring_order_L{L}.txt"), dtype=np.int64, comments="#")
    theta = sampling.equiangular_set(L)[order]
    c = synth.decaying_coeffs(L, 1, SEED)[0]
    t0 = time.time()
    s = osht.inverse(c, L, theta)
    t1 = time.time()
    c_r = osht.forward(s, L, theta)
    t2 = time.time()
    e1max, e1mean = osht.errors_spectral(c, c_r)
    ci, si = indices(L, N_COEF.get(L, 2048), N_SAMP.get(L, 512))
    h = lambda a: hashlib.sha256(np.ascontiguousarray(a).view(np.float64).tobytes()).hexdigest()  # noqa: E731
    path = os.path.join(HERE, f"oracle_L{L}.txt")
    with open(path, "w") as f:
        f.write(f"# oracle reference values, L={L}, written by tests/golden/make_oracle_reference.py\n")
        f.write(f"# input: synth.decaying_coeffs(L, 1, {SEED})[0]; rings: ring_order_L{L}.txt (Eq. (19) set)\n")
        f.write("# s = oracle.sht.inverse(c) (Procedure 2); c_r = oracle.sht.forward(s) (Procedure 1)\n")
        f.write(f"L {L}\nseed {SEED}\n")
        f.write(f"oracle_E1_max {e1max:.17e}\noracle_E1_mean {e1mean:.17e}\n")
        f.write(f"max_abs_s {np.abs(s).max():.17e}\nmax_abs_c {np.abs(c).max():.17e}\n")
        f.write(f"sha256_c_r {h(c_r)}\nsha256_s {h(s)}\n")
        f.write(f"seconds_inverse {t1 - t0:.1f}\nseconds_forward {t2 - t1:.1f}\n")
        for i in ci:
            f.write(f"c {i} {c_r[i].real:.17e} {c_r[i].imag:.17e}\n")
        for i in si:
            f.write(f"s {i} {s[i].real:.17e} {s[i].imag:.17e}\n")
    print(f"L={L}: E1_max {e1max:.3e}, inverse {t1 - t0:.0f} s, forward {t2 - t1:.0f} s -> {path}", flush=True)


def read(L):
    """Parse oracle_L{L}.txt: (header dict, coefficient indices, values, sample indices, values)."""
    hdr, ci, cv, si, sv = {}, [], [], [], []
    with open(os.path.join(HERE, f"oracle_L{L}.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            p = line.split()
            if p[0] == "c":
                ci.append(int(p[1]))
                cv.append(float(p[2]) + 1j * float(p[3]))
            elif p[0] == "s":
                si.append(int(p[1]))
                sv.append(float(p[2]) + 1j * float(p[3]))
            else:
                hdr[p[0]] = p[1]
    return hdr, np.array(ci), np.array(cv), np.array(si), np.array(sv)


if __name__ == "__main__":
    for arg in sys.argv[1:]:
        main(int(arg))
