"""Autograd through the hand-written adjoints, checked by central finite differences and against
the oracle's dense adjoint (the differentiation workload: real signals, loss
||forward(x) - c||^2 + ||inverse(c) - x||^2)."""
import numpy as np
import pytest
import torch

from oracle import sht as osht
from paper_1403_4661_gb300 import synth
from tests.helpers import oracle_thetas

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1403_4661_gb300 import build
    build.build()


def _loss(plan, x, c):
    from paper_1403_4661_gb300 import sht as S
    r1 = S.forward(plan, x) - c
    r2 = S.inverse(plan, c) - x
    return (r1.abs() ** 2).sum() + (r2.abs() ** 2).sum()


@pytest.mark.parametrize("L,B", [(8, 2), (256, 32)])
def test_loss_gradients_by_finite_differences(L, B):
    from paper_1403_4661_gb300.sht import Plan
    p = Plan(L, theta=oracle_thetas(L))
    x = torch.from_numpy(synth.normal_samples(L, B, 1)).to(DEV).requires_grad_(True)
    c = torch.from_numpy(synth.normal_coeffs(L, B, 2)).to(DEV).requires_grad_(True)
    loss = _loss(p, x, c)
    gx, gc = torch.autograd.grad(loss, (x, c))
    rng = np.random.default_rng(3)
    # the loss is exactly quadratic in (x, c), so the central difference equals the directional
    # derivative for any step; a step of 1e-2 keeps the cancellation error (|loss| u / h) far below
    # the tolerance, where 1e-6 left it within a factor of 2 at L = 256
    h = 1e-2
    for _ in range(8 if L > 64 else 16):
        dx = torch.from_numpy(rng.standard_normal(x.shape)).to(DEV)
        dc = torch.from_numpy(rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).to(DEV)
        with torch.no_grad():
            fd = (_loss(p, x + h * dx, c + h * dc) - _loss(p, x - h * dx, c - h * dc)) / (2 * h)
        # PyTorch's complex gradient is conj(dL/dz*)*2-convention: directional derivative = Re<g, d>
        an = (gx * dx).sum() + (gc.conj() * dc).real.sum()
        assert abs(fd.item() - an.item()) <= 1e-6 * max(1.0, abs(an.item()))


def test_backward_equals_dense_oracle_adjoint():
    from paper_1403_4661_gb300 import sht as S
    from paper_1403_4661_gb300.sht import Plan
    L = 10
    th = oracle_thetas(L)
    A = osht.dense_matrix(L, th)
    p = Plan(L, theta=th)
    s = torch.from_numpy(synth.uniform_samples(L, 1, 5)).to(DEV).requires_grad_(True)
    w = synth.normal_coeffs(L, 1, 6)
    out = S.forward(p, s)
    (g,) = torch.autograd.grad(out, s, grad_outputs=torch.from_numpy(w).to(DEV))
    np.testing.assert_allclose(g.cpu().numpy(), osht.dense_forward_adjoint(w, A), atol=1e-11)
    c = torch.from_numpy(synth.normal_coeffs(L, 1, 7)).to(DEV).requires_grad_(True)
    y = synth.uniform_samples(L, 1, 8)
    out = S.inverse(p, c)
    (g,) = torch.autograd.grad(out, c, grad_outputs=torch.from_numpy(y).to(DEV))
    np.testing.assert_allclose(g.cpu().numpy(), osht.dense_inverse_adjoint(y, A), atol=1e-11)
