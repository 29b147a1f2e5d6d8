"""SHT_F32 plans (every step in float32, complex64 signals) against the oracle.

Tolerances: 1e-4 relative to the largest coefficient (forward) or sample (inverse).  A float32
emulation of the bin-space algorithm on the oracle's tables gives 2e-7 (L = 16) to 2.3e-6
(L = 129) for the forward: the float32 rounding (6e-8) amplified as float64 rounding is in the
float64 path.  The oracle is fed the complex64 inputs themselves (widened exactly), so only the
arithmetic is compared.  Adjoints: dot-product identities 1e-5 relative; the differentiation
workload (32 real signals at L = 256) by central finite differences, 1e-2 relative.
"""
import numpy as np
import pytest
import torch

from oracle import sht as osht
from paper_1403_4661_gb300 import synth
from tests.helpers import oracle_thetas

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1403_4661_gb300 import build
    build.build()


def _plan(L):
    from paper_1403_4661_gb300.sht import Plan
    return Plan(L, theta=oracle_thetas(L), dtype="f32")


def _c64(x):
    return np.ascontiguousarray(x).astype(np.complex64)


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


SIZES = [(1, 1), (3, 1), (31, 2), (33, 2), (65, 3), (130, 1)]


@pytest.mark.parametrize("L,B", SIZES)
def test_f32_inverse_matches_oracle(L, B):
    c = _c64(synth.uniform_coeffs(L, B, 300 + L))
    ref = osht.inverse(c.astype(np.complex128), L, oracle_thetas(L))
    got = _plan(L).inverse(_gpu(c))
    assert got.dtype == torch.complex64
    err = np.abs(got.cpu().numpy().astype(np.complex128) - ref).max()
    print(f"L={L} inverse f32 err {err:.2e} (max |s| {np.abs(ref).max():.2f})")
    assert err <= TOL * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("L,B", SIZES)
def test_f32_forward_matches_oracle(L, B):
    s = _c64(synth.uniform_samples(L, B, 400 + L))
    ref = osht.forward(s.astype(np.complex128), L, oracle_thetas(L))
    got = _plan(L).forward(_gpu(s))
    assert got.dtype == torch.complex64
    err = np.abs(got.cpu().numpy().astype(np.complex128) - ref).max()
    print(f"L={L} forward f32 err {err:.2e} (max |f| {np.abs(ref).max():.2f})")
    assert err <= TOL * max(1.0, np.abs(ref).max())


def test_f32_plan_takes_complex64_only():
    p = _plan(8)
    with pytest.raises(TypeError):
        p.forward(torch.zeros(1, 64, dtype=torch.complex128, device=DEV))
    with pytest.raises(TypeError):
        p.inverse(torch.zeros(1, 64, dtype=torch.complex128, device=DEV))


def test_f32_rejected_by_noalloc_and_uneven():
    from paper_1403_4661_gb300 import sht as S
    p = _plan(8)
    x = torch.zeros(1, 64, dtype=torch.complex128, device=DEV)
    with pytest.raises(S.SHTError) as ei:
        S._call("sht_forward_noalloc", p.handle, x, torch.empty_like(x), 1)
    assert ei.value.status == 2  # SHT_ERR_UNSUPPORTED
    with pytest.raises(S.SHTError) as ei:
        S.forward_uneven([p], [0], [0], x)
    assert ei.value.status == 2


@pytest.mark.parametrize("L,B", [(16, 2), (100, 3)])
def test_f32_adjoint_dot_products(L, B):
    """<A x, y> = <x, A^H y> and <F s, w> = <s, F^H w> in float32."""
    p = _plan(L)
    x = _gpu(_c64(synth.normal_coeffs(L, B, 11)))
    y = _gpu(_c64(synth.normal_samples(L, B, 12) + 1j * synth.normal_samples(L, B, 13)))
    lhs = torch.vdot(p.inverse(x).flatten().to(torch.complex128), y.flatten().to(torch.complex128))
    rhs = torch.vdot(x.flatten().to(torch.complex128), p.inverse_adjoint(y).flatten().to(torch.complex128))
    assert abs(lhs - rhs).item() <= 1e-5 * abs(lhs).item()
    w = x
    s = y
    lhs = torch.vdot(p.forward(s).flatten().to(torch.complex128), w.flatten().to(torch.complex128))
    rhs = torch.vdot(s.flatten().to(torch.complex128), p.forward_adjoint(w).flatten().to(torch.complex128))
    assert abs(lhs - rhs).item() <= 1e-5 * abs(lhs).item()


def test_f32_backward_matches_dense_oracle_adjoint():
    from paper_1403_4661_gb300 import sht as S
    L = 10
    th = oracle_thetas(L)
    A = osht.dense_matrix(L, th)
    p = _plan(L)
    s = _gpu(_c64(synth.uniform_samples(L, 1, 5))).requires_grad_(True)
    w = _c64(synth.normal_coeffs(L, 1, 6))
    (g,) = torch.autograd.grad(S.forward(p, s), s, grad_outputs=_gpu(w))
    ref = osht.dense_forward_adjoint(w.astype(np.complex128), A)
    assert np.abs(g.cpu().numpy() - ref).max() <= TOL * max(1.0, np.abs(ref).max())
    c = _gpu(_c64(synth.normal_coeffs(L, 1, 7))).requires_grad_(True)
    y = _c64(synth.uniform_samples(L, 1, 8))
    (g,) = torch.autograd.grad(S.inverse(p, c), c, grad_outputs=_gpu(y))
    ref = osht.dense_inverse_adjoint(y.astype(np.complex128), A)
    assert np.abs(g.cpu().numpy() - ref).max() <= TOL * max(1.0, np.abs(ref).max())


def test_f32_loss_gradients_by_finite_differences():
    """The differentiation workload in float32: 32 real signals at L = 256,
    loss = ||forward(x) - c||^2 + ||inverse(c) - x||^2 (norms summed in float64)."""
    from paper_1403_4661_gb300 import sht as S
    L, B = 256, 32
    p = _plan(L)
    x = torch.from_numpy(synth.normal_samples(L, B, 1)).to(DEV).float().requires_grad_(True)
    c = _gpu(_c64(synth.normal_coeffs(L, B, 2))).requires_grad_(True)

    def loss(x, c):
        r1 = (S.forward(p, x) - c).to(torch.complex128)
        r2 = (S.inverse(p, c) - x).to(torch.complex128)
        return (r1.abs() ** 2).sum() + (r2.abs() ** 2).sum()

    gx, gc = torch.autograd.grad(loss(x, c), (x, c))
    rng = np.random.default_rng(3)
    h = 1e-1   # the loss is quadratic: the central difference is exact up to rounding for any step
    for _ in range(8):
        dx = torch.from_numpy(rng.standard_normal(x.shape)).to(DEV).float()
        dc = _gpu(_c64(rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)))
        with torch.no_grad():
            fd = (loss(x + h * dx, c + h * dc) - loss(x - h * dx, c - h * dc)) / (2 * h)
        an = (gx.double() * dx.double()).sum() + (gc.conj().to(torch.complex128) * dc.to(torch.complex128)).real.sum()
        assert abs(fd.item() - an.item()) <= 1e-2 * max(1.0, abs(an.item()))
