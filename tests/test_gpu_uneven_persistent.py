"""Uneven batches in one persistent launch per direction (sht_uneven_create / _forward / _inverse)
vs the oracle, signal by signal, on the uneven-batch workload (L log-uniform, f_lm re/im uniform
[-1, 1]) at band-limits the oracle covers in seconds; edge cases L = 1, 2 and the direct / chirp-z
ring boundary (k = 31 / 32); agreement with the per-plan grouped calls; graph capture."""
import numpy as np
import pytest
import torch

from oracle import sht as osht
from paper_1403_4661_gb300 import synth
from tests.helpers import oracle_thetas, tol_samples

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1403_4661_gb300 import build
    build.build()


def _workload(Ls, seed, dtypes=("f64", "f64_tensor")):
    """Plans (one per distinct L, arithmetic alternating), a shuffled packing with gaps."""
    from paper_1403_4661_gb300.sht import Plan
    distinct = sorted(set(int(L) for L in Ls))
    plans = [Plan(L, theta=oracle_thetas(L), dtype=dtypes[i % len(dtypes)]) for i, L in enumerate(distinct)]
    index = [distinct.index(int(L)) for L in Ls]
    order = np.random.default_rng(seed).permutation(len(Ls))
    offsets = np.zeros(len(Ls), dtype=np.int64)
    pos = 3   # a gap before the first signal and between signals
    for i in order:
        offsets[i] = pos
        pos += int(Ls[i]) ** 2 + 1
    coeffs = [synth.uniform_coeffs(int(L), 1, seed * 1000 + i)[0] for i, L in enumerate(Ls)]
    packed = np.zeros(pos, dtype=np.complex128)
    for i, c in enumerate(coeffs):
        packed[offsets[i]:offsets[i] + c.size] = c
    return plans, index, offsets, coeffs, packed


@pytest.mark.parametrize("Ls", [
    list(synth.loguniform_bandlimits(24, 8, 96, 7)),
    [1, 2, 31, 32, 33, 64, 65, 3],
])
def test_persistent_uneven_matches_oracle(Ls):
    from paper_1403_4661_gb300.sht import UnevenBatch
    plans, index, offsets, coeffs, packed = _workload(Ls, 7)
    ub = UnevenBatch(plans, index, offsets)
    c = torch.from_numpy(packed).to(DEV)
    s = ub.inverse(c)
    c2 = ub.forward(s)
    ub.check()
    s_h, c2_h = s.cpu().numpy(), c2.cpu().numpy()
    for i, L in enumerate(Ls):
        L = int(L)
        sl = slice(int(offsets[i]), int(offsets[i]) + L * L)
        th = oracle_thetas(L)
        ref = osht.inverse(coeffs[i][None], L, th)[0]
        assert np.abs(s_h[sl] - ref).max() <= tol_samples(ref), (i, L)
        ref_f = osht.forward(s_h[sl][None], L, th)[0]
        assert np.abs(c2_h[sl] - ref_f).max() <= 1e-11, (i, L)
        assert np.abs(c2_h[sl] - coeffs[i]).max() <= 1e-11, (i, L)
    ub.close()


def test_persistent_uneven_agrees_with_grouped_calls_and_replays_in_a_graph():
    from paper_1403_4661_gb300.sht import UnevenBatch, forward_uneven, inverse_uneven
    Ls = list(synth.loguniform_bandlimits(16, 16, 130, 11))
    plans, index, offsets, coeffs, packed = _workload(Ls, 11)
    ub = UnevenBatch(plans, index, offsets)
    c = torch.from_numpy(packed).to(DEV)
    # outputs zeroed first: the gaps between the signals are written by neither call
    s_ref = inverse_uneven(plans, index, offsets, c, out=torch.zeros_like(c))
    c_ref = forward_uneven(plans, index, offsets, s_ref, out=torch.zeros_like(c))
    s = torch.zeros_like(c)
    c2 = torch.zeros_like(c)
    ub.inverse(c, out=s)
    ub.forward(s, out=c2)
    torch.cuda.synchronize()
    scale = max(1.0, float(s_ref.abs().max()))
    assert float((s - s_ref).abs().max()) <= 1e-11 * scale
    assert float((c2 - c_ref).abs().max()) <= 1e-11
    # the same two launches captured in a CUDA graph and replayed: bit-identical
    s_g = torch.zeros_like(c)
    c_g = torch.zeros_like(c)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            ub.inverse(c, out=s_g)
            ub.forward(s_g, out=c_g)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    ub.check()
    assert torch.equal(s_g, s) and torch.equal(c_g, c2)
    ub.close()


def test_persistent_uneven_rejects_bad_layouts():
    from paper_1403_4661_gb300.sht import Plan, SHTError, UnevenBatch
    p8 = Plan(8, theta=oracle_thetas(8))
    with pytest.raises(SHTError, match="INVALID_ARG"):
        UnevenBatch([p8], [0, 0], [0, 10])        # overlapping signals (64 elements each)
    with pytest.raises(SHTError, match="INVALID_ARG"):
        UnevenBatch([p8], [1], [0])               # plan index out of range
    with pytest.raises(SHTError, match="INVALID_ARG"):
        UnevenBatch([p8], [0], [-1])              # negative offset
    f32 = Plan(8, theta=oracle_thetas(8), dtype="f32")
    with pytest.raises(SHTError, match="UNSUPPORTED"):
        UnevenBatch([f32], [0], [0])
    ub = UnevenBatch([p8], [0], [0])
    x = torch.zeros(64, dtype=torch.complex128, device=DEV)
    with pytest.raises(SHTError, match="INVALID_ARG"):
        ub._run("sht_uneven_forward", x, x, None)  # input and output overlap
    ub.close()


def test_table_free_plans_regenerate_ptilde():
    """Plans made with SHT_PLAN_NO_PTILDE drop the L^3/2 P~ table; the persistent launches rebuild
    P~ by its recursion and give the oracle's results, and agree with table-holding plans."""
    from paper_1403_4661_gb300.sht import Plan, SHTError, UnevenBatch
    Ls = [1, 2, 40, 130, 77, 130]
    plans_t, index, offsets, coeffs, packed = _workload(Ls, 13, dtypes=("f64",))
    distinct = sorted(set(Ls))
    plans_f = [Plan(L, theta=oracle_thetas(L), keep_ptilde=False) for L in distinct]
    assert plans_f[-1].info()["table_bytes"] < plans_t[-1].info()["table_bytes"]
    c = torch.from_numpy(packed).to(DEV)
    ut, uf = UnevenBatch(plans_t, index, offsets), UnevenBatch(plans_f, index, offsets)
    s_t, s_f = ut.inverse(c), uf.inverse(c)
    c_t, c_f = ut.forward(s_t), uf.forward(s_f)
    uf.check()
    scale = max(1.0, float(s_t.abs().max()))
    assert float((s_f - s_t).abs().max()) <= 1e-13 * scale
    assert float((c_f - c_t).abs().max()) <= 1e-12
    s_h, c_h = s_f.cpu().numpy(), c_f.cpu().numpy()
    for i, L in enumerate(Ls):
        sl = slice(int(offsets[i]), int(offsets[i]) + L * L)
        ref = osht.inverse(coeffs[i][None], L, oracle_thetas(L))[0]
        assert np.abs(s_h[sl] - ref).max() <= tol_samples(ref), (i, L)
        assert np.abs(c_h[sl] - coeffs[i]).max() <= 1e-11, (i, L)
    # the batched entry points refuse a plan without its P~ table
    with pytest.raises(SHTError, match="UNSUPPORTED"):
        plans_f[-1].forward(torch.zeros((1, 130 * 130), dtype=torch.complex128, device=DEV))
    with pytest.raises(SHTError, match="UNSUPPORTED"):
        Plan(16, keep_ptilde=False, dtype="f64_tensor")
    ut.close()
    uf.close()
