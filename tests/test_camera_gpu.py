"""Camera side on the device (cbp_encrypt) against the oracle (Section 3):
the per-frame kernels bit-exact (the same Philox-4x32-10 words, the same
normalisation order), the accepted draw indices identical (the coprimality
decisions, taken far from the tolerance), the blurred streams and the
cascaded pair within the forward model's float bounds, and Eq. 4's identity
on the device's outputs."""
import numpy as np
import pytest
import torch
from scipy.signal import convolve2d

import oracle
from oracle import camera
from tests._inputs import rel

pytestmark = pytest.mark.gpu


def test_kernels_streams_and_cascade_match_the_oracle(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    rng = np.random.default_rng(17)
    lat = rng.uniform(size=(3, 2, 30, 34))
    out = cbp.cbp_encrypt(gpu_ctx, torch.from_numpy(lat).cuda(), 7, 5, seed=99, frame0=3, cascade=(3, 4))
    for f in range(3):
        o = camera.encrypt(lat[f], 99, 3 + f, 7, 5, cascade=(3, 4))
        assert np.array_equal(out["k1"][f].cpu().numpy(), o["k1"])
        assert np.array_equal(out["k2"][f].cpu().numpy(), o["k2"])
        assert np.array_equal(out["k3"][f].cpu().numpy(), o["k3"])
        assert np.array_equal(out["k4"][f].cpu().numpy(), o["k4"])
        assert out["attempts"][f] == o["attempt"] and out["attempts"][3 + f] == o["attempt_cascade"]
        for key in ("b1", "b2", "c1", "c2"):
            assert rel(out[key][f].cpu().numpy(), o[key]) <= 1e-14, key
    # Eq. 4 on the device's own outputs: b1 (x) k2 = b2 (x) k1
    b1, b2 = out["b1"][0, 0].cpu().numpy(), out["b2"][0, 0].cpu().numpy()
    k1, k2 = out["k1"][0].cpu().numpy(), out["k2"][0].cpu().numpy()
    assert rel(convolve2d(b1, k2), convolve2d(b2, k1)) <= 1e-13


def test_redraw_decisions_match_the_oracle(gpu_ctx):
    """A strict tolerance makes most draws fail: the device redraws exactly
    as the oracle does, and gives up (-1) where it does."""
    from paper_1203_4874_gb300 import cbp
    rng = np.random.default_rng(5)
    lat = rng.uniform(size=(12, 1, 16, 16))
    out = cbp.cbp_encrypt(gpu_ctx, torch.from_numpy(lat).cuda(), 5, 5, seed=123, tol=3e-3, max_attempts=4)
    want = [camera.draw_pair(123, f, 5, 5, 5, max_attempts=4, tol=3e-3)[2] for f in range(12)]
    assert out["attempts"] == want
    assert any(a > 0 for a in want) and len(set(want)) > 1


def test_float_frames_and_noise(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    rng = np.random.default_rng(6)
    lat = rng.uniform(size=(2, 1, 40, 44)).astype(np.float32)
    out = cbp.cbp_encrypt(gpu_ctx, torch.from_numpy(lat).cuda(), 15, 17, seed=7)
    for f in range(2):
        ref = oracle.blur_full(lat[f, 0].astype(np.float64), out["k1"][f].cpu().numpy())
        assert rel(out["b1"][f, 0].double().cpu().numpy(), ref) <= 2e-6
    noisy = cbp.cbp_encrypt(gpu_ctx, torch.from_numpy(lat).cuda(), 15, 17, seed=7, sigma=1e-3)
    d = (noisy["b1"] - out["b1"]).double().cpu().numpy()
    assert abs(d.mean()) < 1e-4 and abs(d.std() / 1e-3 - 1) < 0.05
