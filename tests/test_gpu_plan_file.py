"""A plan's co-latitudes saved and loaded (sht_plan_save / sht_plan_load): the loaded plan has the
same rings and gives bit-identical transforms, for the float64 and the tensor-core arithmetic."""
import numpy as np
import pytest
import torch

from paper_1403_4661_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1403_4661_gb300 import build
    build.build()


@pytest.mark.parametrize("dtype", ["f64", "f64_tensor"])
def test_saved_rings_rebuild_the_same_plan(dtype, tmp_path):
    from paper_1403_4661_gb300.sht import Plan
    L, B = 48, 2
    p = Plan(L, dtype=dtype)                  # the library's greedy ordering
    path = tmp_path / f"rings_L{L}.bin"
    p.save(path)
    q = Plan.load(path, dtype=dtype)
    assert q.L == L
    np.testing.assert_array_equal(q.theta, p.theta)
    s = torch.from_numpy(synth.uniform_samples(L, B, 9)).to(DEV)
    c = torch.from_numpy(synth.uniform_coeffs(L, B, 10)).to(DEV)
    assert torch.equal(p.forward(s), q.forward(s))
    assert torch.equal(p.inverse(c), q.inverse(c))
