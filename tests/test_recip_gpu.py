"""The eigen-solver's double-precision reciprocal and reciprocal square root
(Newton-Raphson from a single-precision seed, two steps) against 1 / x and
1 / sqrt(x) across the exponent range, up to the 1e+-30 guards and beyond
them (where plain division and sqrt take over).

Bounds (u = 2^-53 = 1.1e-16): after two steps the iteration's own error is
below double rounding, so each result carries the rounding of its last step's
few operations, at most ~2 ulp (4.4e-16).  The checks add their own rounding:
r x - 1 one multiplication (0.5 ulp) -> 4e-16 in all; for 1 / sqrt(x) the
reference's sqrt and division (up to 1 ulp) and the comparing division (0.5
ulp) -> 8e-16."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_reciprocals_match_division_and_sqrt(built_lib):
    from paper_1203_4874_gb300 import cbp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(0)
    e = rng.uniform(-40, 40, size=200000)
    x = rng.uniform(1, 10, size=e.size) * 10.0 ** e
    x[::2] *= -1
    x[:8] = [1e-30, 1.0000001e-30, 9.999999e29, 1e30, -1e-30, 2.0 ** -100, 2.0 ** 100, 1.0]
    X = torch.from_numpy(x).cuda()
    r = torch.empty_like(X)
    q = torch.empty_like(X)
    assert cbp.lib().cbp_check_recip(X.data_ptr(), X.numel(), r.data_ptr(), q.data_ptr(), None) == 0
    torch.cuda.synchronize()
    r, q = r.cpu().numpy(), q.cpu().numpy()
    assert np.max(np.abs(r * x - 1.0)) <= 4e-16
    pos = x > 0
    ref = 1.0 / np.sqrt(x[pos])
    assert np.max(np.abs(q[pos] / ref - 1.0)) <= 8e-16
    assert np.all(q[~pos] == 0.0)
