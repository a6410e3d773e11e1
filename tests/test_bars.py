"""CPU checks of the tolerance derivations the GPU parity bars rely on.

The MIXED bars add mixed_position_bound(x) (tests.gpu_util): rounding every
coordinate to FP32 (u |x| per coordinate, u = 2^-24) moves a pair
separation by at most 2 sqrt(3) u |x|max, which changes the pair's r^-12
term by at most 12 * 2 sqrt(3) u |x|max / r_min of itself to first order.
Here the exact FP32 rounding of real configurations is applied and the
largest relative change of any pair's r^-12 term is compared with it."""
import numpy as np
import pytest
from scipy.spatial.distance import pdist

from paper_1810_03358_gb300 import synth
from tests.gpu_util import U32, mixed_position_bound


@pytest.mark.parametrize("n,seed", [(60, 3), (200, 11), (700, 1400)])
def test_position_bound_covers_fp32_rounding(n, seed):
    x = synth.make_system(n, seed).x
    x32 = x.astype(np.float32).astype(np.float64)
    d, d32 = pdist(x), pdist(x32)
    rel = np.abs((d32 / d) ** -12 - 1.0).max()
    bound = mixed_position_bound(x)
    # first order in the tiny relative move (<1e-5): the second-order term
    # adds (1 + 13 eps / 2) at most
    assert rel <= bound * (1.0 + 1e-3), (rel, bound)
    # and the bound is not vacuous: within two orders of magnitude of the
    # worst pair's actual change
    assert bound <= 100.0 * rel, (rel, bound)


def test_fp32_unit_roundoff():
    assert U32 == np.finfo(np.float32).eps / 2
    x = np.float64(1.0) + U32
    assert np.float32(x) == np.float32(1.0)  # ties to even at 1 + u
