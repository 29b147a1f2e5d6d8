"""Plans on the ring sets of the alternative measures (Sec. III-F, SHT_MEASURE_SIN / _TAN13): the
library's rings (closed forms, ordered by the GPU planner) equal the oracle's (numerical
integration of the measures, oracle orderings); the inverse matches the oracle; the round trip
closes within 1e-12 x the largest condition number of the P_m (these sets are ill-conditioned by
design: at L = 12 the oracle itself differs from dense brute force by up to 4e-14 x that number)."""
import numpy as np
import pytest
import torch

from oracle import sampling
from oracle import sht as osht
from paper_1403_4661_gb300 import synth
from tests.helpers import tol_samples

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore")]
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1403_4661_gb300 import build
    build.build()


@pytest.mark.parametrize("measure", ["sin", "tan13"])
@pytest.mark.parametrize("ordering", ["simple", "greedy"])
def test_alternative_measure_plans(measure, ordering):
    from paper_1403_4661_gb300.sht import Plan
    L, B = 12, 2
    p = Plan(L, ordering=ordering, measure=measure)
    ref = sampling.thetas(L, ordering, measure)
    np.testing.assert_allclose(p.theta, ref, atol=1e-13, rtol=0)
    kmax = sampling.order_conditions(L, ref).max()
    c = synth.uniform_coeffs(L, B, 40)
    s = p.inverse(torch.from_numpy(c).to(DEV))
    s_ref = osht.inverse(c, L, ref)
    assert np.abs(s.cpu().numpy() - s_ref).max() <= tol_samples(s_ref)
    c2 = p.forward(s).cpu().numpy()
    assert np.abs(c2 - c).max() <= 1e-12 * kmax
