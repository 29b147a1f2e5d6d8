"""Host-side helpers of bench.py: the sampled comparison with the stored oracle values and the
DRAM-traffic record lookup (valid only for the captured kernel source)."""
import importlib.util
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _golden(L):
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        import make_oracle_reference as m
        return m.read(L)
    finally:
        sys.path.pop(0)


def test_vs_stored_oracle_reads_the_stored_signal():
    b = _bench()
    L = 1024
    hdr, ci, cv, si, sv = _golden(L)
    s = torch.zeros(2, L * L, dtype=torch.complex128)
    c2 = torch.zeros_like(s)
    s[0, si] = torch.from_numpy(sv)
    c2[0, ci] = torch.from_numpy(cv)
    r = b._vs_stored_oracle(L, 1000, s, c2)
    assert r["coeff_max_abs_diff"] == 0.0 and r["sample_max_rel_diff"] == 0.0
    assert r["n_coeff"] == len(ci) and r["n_sample"] == len(si)
    # a perturbed coefficient shows up at its size; other seeds and sizes have no record
    c2[0, ci[3]] += 1e-9
    assert abs(b._vs_stored_oracle(L, 1000, s, c2)["coeff_max_abs_diff"] - 1e-9) < 1e-12
    assert b._vs_stored_oracle(L, 1001, s, c2) is None
    assert b._vs_stored_oracle(24, 1000, s, c2) is None


def test_traffic_record_follows_the_source_hash():
    b = _bench()
    rec = {}
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        parts = dict(p.split("=", 1) for p in line.split() if "=" in p)
        if parts.get("kernel") == "chain_tc" and parts.get("L") == "1024" and parts.get("batch") == "64":
            rec = parts
    tr, note = b._traffic("chain_tc", 1024, 64, "chain.cu")
    if rec and rec["src_sha"] == b._src_hash("chain.cu"):
        assert tr == float(rec["dram_bytes_per_launch"])      # the record of this very source
    else:
        assert tr is None                                      # no record, or a stale one
    assert b._traffic("chain_tc", 1024, 65, "chain.cu")[0] is None
    tr2, note2 = b._traffic("chain_tc", 1024, 64, "tc_gemm.cu")   # another file's hash: stale
    assert tr2 is None and ("stale" in note2 or not rec)
