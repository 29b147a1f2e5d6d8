"""Spin-s transforms (Sec. III-H, Appendix A) through the C ABI against the spin oracle.

Inverse (a plain sum): element by element at L up to 128, s = 1, 2, -1, 1e-11 relative to the
largest sample.  Inverse adjoint: the dense conjugate transpose of the oracle's explicit-sum
matrix at L = 8, and the dot-product identity <A c, y> = <c, A^H y> at L = 64.
Forward (Procedure 1): against the oracle's forward at small L, tolerance max(1e-11, 4 x the
oracle's own round-trip error on that input): the order-by-order elimination amplifies rounding
far more for s != 0 than for s = 0 (the oracle shows the same), so the forward is checked only
where it is accurate.
"""
import numpy as np
import pytest
import torch

from oracle import sampling, spin
from paper_1403_4661_gb300 import synth
from tests.helpers import tol_samples

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1403_4661_gb300 import build
    build.build()


def _plan(L, s):
    from paper_1403_4661_gb300.sht import Plan
    return Plan(L, theta=sampling.thetas(L, "greedy"), spin=s)


def _coeffs(L, B, seed, s):
    c = synth.uniform_coeffs(L, B, seed)
    c[:, : s * s] = 0.0
    return c


@pytest.mark.parametrize("L,s,B", [(3, 1, 1), (8, 2, 2), (33, 1, 2), (64, -1, 1), (100, 2, 1), (128, 1, 1)])
def test_spin_inverse_matches_oracle(L, s, B):
    th = sampling.thetas(L, "greedy")
    c = _coeffs(L, B, 300 + L, s)
    ref = spin.inverse(c, L, th, s)
    p = _plan(L, s)
    got = p.inverse(torch.from_numpy(c).to(DEV)).cpu().numpy()
    assert np.abs(got - ref).max() <= tol_samples(ref)
    # coefficients of degrees below |s| are ignored on input
    c2 = c.copy()
    c2[:, : s * s] = 5.0
    got2 = p.inverse(torch.from_numpy(c2).to(DEV)).cpu().numpy()
    assert np.array_equal(got, got2)


@pytest.mark.parametrize("s", [1, 2])
def test_spin_inverse_adjoint_dense(s):
    L = 8
    th = sampling.thetas(L, "greedy")
    A = spin.dense_matrix(L, th, s)
    y = synth.uniform_samples(L, 2, 9)
    p = _plan(L, s)
    got = p.inverse_adjoint(torch.from_numpy(y).to(DEV)).cpu().numpy()
    ref = y @ A.conj()
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_spin_inverse_adjoint_dot_product():
    L, s = 64, 2
    th = sampling.thetas(L, "greedy")
    c = _coeffs(L, 1, 4, s)[0]
    y = synth.uniform_samples(L, 1, 5)[0]
    p = _plan(L, s)
    Ac = spin.inverse(c, L, th, s)
    AHy = p.inverse_adjoint(torch.from_numpy(y[None]).to(DEV)).cpu().numpy()[0]
    lhs, rhs = np.vdot(y, Ac), np.vdot(AHy, c)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("L,s", [(2, 1), (4, 1), (6, 2), (8, 1), (8, 2), (10, -1), (12, 1)])
def test_spin_forward_matches_oracle(L, s):
    th = sampling.thetas(L, "greedy")
    c = _coeffs(L, 2, 700 + L, s)
    x = spin.inverse(c, L, th, s)
    ref = spin.forward(x, L, th, s)
    tol = max(1e-11, 4.0 * float(np.abs(ref - c).max()))
    p = _plan(L, s)
    got = p.forward(torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.abs(got - ref).max() <= tol
    assert np.abs(got - c).max() <= tol
    assert np.all(got[:, : s * s] == 0)


def test_spin_plan_refusals():
    from paper_1403_4661_gb300.sht import Plan, SHTError

    with pytest.raises(SHTError, match="UNSUPPORTED"):
        Plan(16, spin=1, dtype="f64_tensor")
    with pytest.raises(SHTError, match="INVALID_ARG"):
        Plan(2, spin=2)
    with pytest.raises(SHTError, match="UNSUPPORTED"):
        Plan(16, spin=9)
    p = _plan(8, 1)
    assert p.info()["spin"] == 1
    x = torch.zeros((1, 64), dtype=torch.complex128, device=DEV)
    with pytest.raises(SHTError, match="UNSUPPORTED"):
        p.forward_adjoint(x)
