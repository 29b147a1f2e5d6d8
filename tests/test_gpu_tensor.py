"""SHT_F64_TENSOR plans (contractions on the BF16 tensor cores from exact slices) vs the oracle.

Same tolerances as the float64 path: coefficients 1e-11 absolute, samples 1e-11 relative to the
largest sample.
"""
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


def _plan(L):
    from paper_1403_4661_gb300.sht import Plan
    return Plan(L, theta=oracle_thetas(L), dtype="f64_tensor")


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


SIZES = [(1, 1), (2, 2), (7, 3), (31, 2), (33, 1), (64, 2), (129, 3), (200, 1)]


@pytest.mark.parametrize("L,B", SIZES)
def test_tensor_inverse_matches_oracle(L, B):
    th = oracle_thetas(L)
    c = synth.uniform_coeffs(L, B, 500 + L)
    ref = osht.inverse(c, L, th)
    p = _plan(L)
    got = p.inverse(_gpu(c)).cpu().numpy()
    p.check()
    assert np.abs(got - ref).max() <= tol_samples(ref)


@pytest.mark.parametrize("L,B", SIZES)
def test_tensor_forward_matches_oracle(L, B):
    th = oracle_thetas(L)
    s = synth.uniform_samples(L, B, 600 + L)
    ref = osht.forward(s, L, th)
    p = _plan(L)
    got = p.forward(_gpu(s)).cpu().numpy()
    p.check()
    assert np.abs(got - ref).max() <= 1e-11


@pytest.mark.parametrize("L,B", [(512, 256), (1024, 64)])
def test_tensor_full_size_sampled(L, B):
    th = oracle_thetas(L)
    c = synth.decaying_coeffs(L, B, 7)
    p = _plan(L)
    cg = _gpu(c)
    s = p.inverse(cg)
    c2 = p.forward(s)
    p.check()
    rng = np.random.default_rng(L + 1)
    idx = np.sort(rng.choice(L * L, 24, replace=False))
    idx[0], idx[-1] = 0, L * L - 1
    sig = [0, B - 1]
    s_h = s[sig].cpu().numpy()
    assert np.abs(s_h[:, idx] - osht.evaluate_samples(c[sig], L, th, idx)).max() <= tol_samples(s_h)
    err = (c2 - cg).abs().max().item()
    assert err <= 1e-11, err
    c2_h = c2[sig[:1]].cpu().numpy()
    assert np.abs(osht.evaluate_samples(c2_h, L, th, idx) - s_h[:1, idx]).max() <= tol_samples(s_h)


def test_tensor_agrees_with_float64_path():
    from paper_1403_4661_gb300.sht import Plan
    L, B = 300, 4
    th = oracle_thetas(L)
    p64, ptc = Plan(L, theta=th), Plan(L, theta=th, dtype="f64_tensor")
    c = _gpu(synth.decaying_coeffs(L, B, 3))
    s64, stc = p64.inverse(c), ptc.inverse(c)
    assert (s64 - stc).abs().max().item() <= 1e-12 * s64.abs().max().item() * 10
    f64, ftc = p64.forward(s64), ptc.forward(s64)
    ptc.check()
    assert (f64 - ftc).abs().max().item() <= 1e-12


def test_tensor_deterministic_and_adjoint():
    L, B = 150, 2
    p = _plan(L)
    x = _gpu(synth.uniform_samples(L, B, 5))
    a, b = p.forward(x), p.forward(x)
    assert torch.equal(a, b)
    y = _gpu(synth.normal_coeffs(L, B, 6))
    lhs = torch.vdot(y.flatten(), p.forward(x).flatten())
    rhs = torch.vdot(p.forward_adjoint(y).flatten(), x.flatten())
    assert abs(lhs - rhs).item() <= 1e-11 * abs(lhs).item()


def test_tensor_deterministic_and_graph_capture():
    """The forward's order chain (one persistent cooperative launch) gives identical results on
    every call and inside a captured CUDA graph."""
    L, B = 150, 5
    p = _plan(L)
    p.reserve(B)
    c = _gpu(synth.uniform_coeffs(L, B, 77))
    s = torch.empty_like(c)
    c2 = torch.empty_like(c)
    p.inverse(c, out=s)
    p.forward(s, out=c2)
    ref = c2.clone()
    p.forward(s, out=c2)
    assert torch.equal(c2, ref)
    c2.zero_()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            p.inverse(c, out=s)
            p.forward(s, out=c2)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        c2.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(c2, ref)
    p.check()
    assert (ref - c).abs().max().item() <= 1e-11


def test_wait_limit_timeout_is_reported_and_the_plan_recovers():
    """A wait limit of 1 ns makes the tensor kernels' waits (grid barriers, mbarriers) give up at
    once: the call is abandoned with SHT_ERR_TIMEOUT in the status word, the context stays usable
    and the next call at the default limit gives the normal result."""
    from paper_1403_4661_gb300.sht import SHTError
    L, B = 96, 4
    p = _plan(L)
    s = _gpu(synth.uniform_samples(L, B, 3))
    ref = p.forward(s)
    p.check()
    with pytest.raises(SHTError):
        p.set_wait_limit(0.0)
    p.set_wait_limit(1e-9)
    p.forward(s)
    p.inverse(ref)
    with pytest.raises(SHTError, match="TIMEOUT"):
        p.check()
    p.set_wait_limit(1.0)
    assert torch.equal(p.forward(s), ref)
    p.check()
