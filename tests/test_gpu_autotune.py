"""Execution paths per batch size (sht_plan_set_paths) and the autotuner that picks among them
(sht_plan_autotune): every path a plan offers matches the oracle, the autotuned plan still does,
also through the uneven calls and a CUDA graph, and paths a plan does not offer are refused.
Tolerances as in the parity tests: 1e-11 (float64-accurate paths), 1e-10 (refined forward),
1e-4 relative (SHT_F32)."""
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


def _plan(L, dtype):
    from paper_1403_4661_gb300.sht import Plan
    return Plan(L, theta=oracle_thetas(L), dtype=dtype)


def _check(p, L, B, seed):
    th = oracle_thetas(L)
    cd = np.complex64 if p.dtype == 5 else np.complex128
    s = synth.uniform_samples(L, B, seed).astype(cd)
    c = synth.uniform_coeffs(L, B, seed + 1).astype(cd)
    f_ref = osht.forward(s.astype(np.complex128), L, th)
    s_ref = osht.inverse(c.astype(np.complex128), L, th)
    f = p.forward(torch.from_numpy(s).to(DEV)).cpu().numpy().astype(np.complex128)
    y = p.inverse(torch.from_numpy(c).to(DEV)).cpu().numpy().astype(np.complex128)
    if p.dtype == 5:
        assert np.abs(f - f_ref).max() <= 1e-4 * max(1.0, np.abs(f_ref).max())
        assert np.abs(y - s_ref).max() <= 1e-4 * max(1.0, np.abs(s_ref).max())
    else:
        # refined plans: 1e-10, their tolerance in the refinement tests
        assert np.abs(f - f_ref).max() <= (1e-10 if p.dtype in (2, 3, 4) else 1e-11)
        assert np.abs(y - s_ref).max() <= tol_samples(s_ref)


@pytest.mark.parametrize("dtype", ["f64_tensor", "f64", "f32"])
def test_every_offered_path_matches_oracle(dtype):
    L, B = 70, 3
    p = _plan(L, dtype)
    fwd = (["tensor"] if dtype == "f64_tensor" else []) + ["simt"]
    inv = fwd
    for fp in fwd:
        for ip in inv:
            for cap in ([0] if fp == "tensor" else [1, 4, 16]):
                p.set_paths(B, fp, ip, cap)
                _check(p, L, B, 10 + cap)


@pytest.mark.parametrize("dtype", ["f64_tensor", "f64", "f32", "tf32_refined"])
def test_autotune_choice_is_valid_and_exact(dtype):
    L, B = 90, 2
    p = _plan(L, dtype)
    if dtype == "tf32_refined":
        p.set_refinement(30, 1e-11)
    t = p.autotune(B)
    print(dtype, t)
    assert t["inverse_ms"] > 0
    if dtype == "tf32_refined":
        assert t["forward_path"] == "default" and t["forward_ms"] == 0
    else:
        assert t["forward_ms"] > 0
        assert t["forward_path"] in (("tensor", "simt") if dtype == "f64_tensor" else ("simt",))
    _check(p, L, B, 20)


def test_paths_not_offered_are_refused():
    from paper_1403_4661_gb300.sht import SHTError
    p = _plan(16, "f64")
    with pytest.raises(SHTError):
        p.set_paths(1, "tensor", "default")
    with pytest.raises(SHTError):
        p.set_paths(1, "default", "default", 17)
    with pytest.raises(SHTError):
        p.set_paths(0, "default", "default")
    r = _plan(16, "bf16x2_refined")
    with pytest.raises(SHTError):
        r.set_paths(1, "simt", "default")
    r.set_paths(1, "default", "simt")


def test_autotuned_uneven_batch_and_graph_replay():
    """Plans tuned for their group sizes, then one uneven call per direction, replayed in a graph."""
    from paper_1403_4661_gb300 import sht as S
    Ls = [24, 40, 57]
    counts = [3, 1, 2]
    plans = [_plan(L, "f64_tensor") for L in Ls]
    for p, n in zip(plans, counts):
        p.autotune(n)
    idx = [0, 0, 0, 1, 2, 2]
    offs, o = [], 0
    for i in idx:
        offs.append(o)
        o += Ls[i] ** 2
    c = synth.uniform_coeffs(1, o, 30)[:, 0].reshape(1, o)   # o values, flat
    cg = torch.from_numpy(np.ascontiguousarray(c[0])).to(DEV)
    sg = S.inverse_uneven(plans, idx, offs, cg)
    fg = S.forward_uneven(plans, idx, offs, sg)
    out = torch.empty_like(fg)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            S.forward_uneven(plans, idx, offs, sg, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, fg)
    s_np = sg.cpu().numpy()
    f_np = fg.cpu().numpy()
    for i, off in zip(idx, offs):
        L = Ls[i]
        th = oracle_thetas(L)
        ref_s = osht.inverse(c[0, off:off + L * L], L, th)
        assert np.abs(s_np[off:off + L * L] - ref_s).max() <= tol_samples(ref_s)
        ref_f = osht.forward(s_np[off:off + L * L], L, th)
        assert np.abs(f_np[off:off + L * L] - ref_f).max() <= 1e-11
