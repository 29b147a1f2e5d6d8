"""Batches of signals with different band-limits (sht_forward_uneven / sht_inverse_uneven) vs the
oracle, signal by signal: the uneven-batch workload (L log-uniform, f_lm re/im uniform[-1, 1]) at
band-limits the oracle covers in seconds."""
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


def _workload(nsig, lo, hi, seed):
    """Band-limits, the plans (one per distinct L, arithmetic alternating), a shuffled packing."""
    from paper_1403_4661_gb300.sht import Plan
    Ls = synth.loguniform_bandlimits(nsig, lo, hi, seed)
    distinct = sorted(set(int(L) for L in Ls))
    plans = [Plan(L, theta=oracle_thetas(L), dtype="f64_tensor" if i % 2 else "f64")
             for i, L in enumerate(distinct)]
    index = [distinct.index(int(L)) for L in Ls]
    order = np.random.default_rng(seed).permutation(nsig)   # signals of one plan not adjacent
    offsets = np.zeros(nsig, dtype=np.int64)
    pos = 0
    for i in order:
        offsets[i] = pos
        pos += int(Ls[i]) ** 2
    coeffs = [synth.uniform_coeffs(int(L), 1, seed * 1000 + i)[0] for i, L in enumerate(Ls)]
    packed = np.zeros(pos, dtype=np.complex128)
    for i, c in enumerate(coeffs):
        packed[offsets[i]:offsets[i] + c.size] = c
    return Ls, plans, index, offsets, coeffs, packed


def test_uneven_inverse_and_forward_match_oracle():
    from paper_1403_4661_gb300.sht import forward_uneven, inverse_uneven
    Ls, plans, index, offsets, coeffs, packed = _workload(24, 8, 96, 5)
    c = torch.from_numpy(packed).to(DEV)
    s = inverse_uneven(plans, index, offsets, c)
    c2 = forward_uneven(plans, index, offsets, s)
    for p in plans:
        p.check()
    s_h, c2_h = s.cpu().numpy(), c2.cpu().numpy()
    for i, L in enumerate(Ls):
        L = int(L)
        sl = slice(int(offsets[i]), int(offsets[i]) + L * L)
        ref = osht.inverse(coeffs[i][None], L, oracle_thetas(L))[0]
        assert np.abs(s_h[sl] - ref).max() <= tol_samples(ref), (i, L)
        ref_f = osht.forward(s_h[sl][None], L, oracle_thetas(L))[0]
        assert np.abs(c2_h[sl] - ref_f).max() <= 1e-11, (i, L)
        assert np.abs(c2_h[sl] - coeffs[i]).max() <= 1e-11, (i, L)


def test_uneven_equals_batched_calls():
    """Consecutive signals of one plan run in place; the results are those of the batched call."""
    from paper_1403_4661_gb300.sht import Plan, forward_uneven, inverse_uneven
    plans = [Plan(L, theta=oracle_thetas(L), dtype=d) for L, d in ((20, "f64"), (33, "f64_tensor"))]
    b = (3, 2)
    c = [torch.from_numpy(synth.uniform_coeffs(p.L, n, 40 + p.L)).to(DEV) for p, n in zip(plans, b)]
    packed = torch.cat([x.reshape(-1) for x in c])
    index = [0] * b[0] + [1] * b[1]
    offsets = [i * 400 for i in range(b[0])] + [b[0] * 400 + i * 33 * 33 for i in range(b[1])]
    s = inverse_uneven(plans, index, offsets, packed)
    f = forward_uneven(plans, index, offsets, s)
    s_ref = torch.cat([p.inverse(x).reshape(-1) for p, x in zip(plans, c)])
    assert torch.equal(s, s_ref)
    f_ref = torch.cat([p.forward(x.reshape(n, -1)).reshape(-1)
                       for p, x, n in zip(plans, torch.split(s_ref, [b[0] * 400, b[1] * 33 * 33]), b)])
    assert torch.equal(f, f_ref)


def test_uneven_rejects_bad_layouts():
    from paper_1403_4661_gb300.sht import SHTError, Plan, inverse_uneven
    p = Plan(8, theta=oracle_thetas(8))
    x = torch.zeros(256, dtype=torch.complex128, device=DEV)
    with pytest.raises(SHTError):
        inverse_uneven([p], [1], [0], x)          # plan index out of range
    with pytest.raises(SHTError):
        inverse_uneven([p], [0, 0], [0, 32], x)   # overlapping signals
    with pytest.raises(SHTError):
        inverse_uneven([p], [0], [-64], x)        # negative offset
    assert inverse_uneven([p], [], [], x).shape == x.shape   # nothing to do


def test_uneven_graph_capture():
    from paper_1403_4661_gb300.sht import forward_uneven, inverse_uneven
    Ls, plans, index, offsets, coeffs, packed = _workload(10, 8, 40, 9)
    c = torch.from_numpy(packed).to(DEV)
    s = inverse_uneven(plans, index, offsets, c)
    f = forward_uneven(plans, index, offsets, s)   # sizes the staging buffers and workspaces
    ref = f.clone()
    f.zero_()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            inverse_uneven(plans, index, offsets, c, out=s)
            forward_uneven(plans, index, offsets, s, out=f)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, ref)
