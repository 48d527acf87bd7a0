"""Kernel-size estimation on the device (cbp_estimate_size) against the
oracle's scan on the same frames: the estimated sizes must be identical
(an integer decision, taken far from the tolerance on these inputs), and the
singularity ratios must agree wherever both are above the double-precision
floor of the device's eigenvalue route (sqrt of ~1e-16 relative: 1e-8)."""
import numpy as np
import pytest
import torch

import oracle
from cbp_synth import draw_kernel_pair
from tests._inputs import make_batch

pytestmark = pytest.mark.gpu


def _compare(gpu_ctx, b1, b2, t_min, t_max, dtype=torch.float64):
    from paper_1203_4874_gb300 import cbp
    B1 = torch.from_numpy(np.ascontiguousarray(b1)).to(dtype).cuda()
    B2 = torch.from_numpy(np.ascontiguousarray(b2)).to(dtype).cuda()
    t1, t2, found, r = cbp.cbp_estimate_size(gpu_ctx, B1, B2, t_min, t_max, 1e-6)
    n = B1.shape[0] if B1.dim() == 4 else 1
    for i in range(n):
        x1 = b1[i] if b1.ndim == 4 else b1
        x2 = b2[i] if b2.ndim == 4 else b2
        if dtype == torch.float32:
            x1 = x1.astype(np.float32).astype(np.float64)
            x2 = x2.astype(np.float32).astype(np.float64)
        o1, o2, ofound, orat = oracle.estimate_size(x1, x2, t_min, t_max, 1e-6)
        assert (t1[i], t2[i], found[i]) == (o1, o2, ofound), (i, t1[i], o1)
        g = r[i].numpy()
        for k, tp in enumerate(range(t_min, t_min + len(g))):
            if tp not in orat:
                assert g[k] < 0
                continue
            if orat[tp] > 1e-6:
                assert abs(g[k] - orat[tp]) <= 1e-6 * orat[tp], (tp, g[k], orat[tp])
            else:
                assert g[k] <= 1e-7, (tp, g[k], orat[tp])
    return t1, t2, found


def test_size_64_noise_free(gpu_ctx):
    b1, b2, *_ = make_batch("single_64", [0], fast=False)
    t1, t2, found = _compare(gpu_ctx, b1, b2, 1, 12)
    assert (t1[0], t2[0], found[0]) == (5, 5, True)


def test_size_480p_noise_free_float_frames(gpu_ctx):
    b1, b2, *_ = make_batch("video_480p", [0], noise=False)
    t1, t2, found = _compare(gpu_ctx, b1, b2, 1, 16, torch.float32)
    assert (t1[0], t2[0], found[0]) == (9, 11, True)


def test_size_batch_of_different_sizes(gpu_ctx):
    """One call over pairs whose kernels differ in size: each pair's estimate
    is its own (the blurred sizes, and so d = t1 - t2, are shared)."""
    rng = np.random.default_rng(41)
    b1s, b2s, truth = [], [], []
    for t in (5, 9, 13):
        lat = rng.uniform(size=(2, 50 - t, 56 - t))      # same blurred size for every pair
        k1, k2 = draw_kernel_pair(rng, t, t, t)
        b1, b2 = oracle.blur_pair(lat, k1, k2)
        b1s.append(b1)
        b2s.append(b2)
        truth.append(t)
    t1, _, found = _compare(gpu_ctx, np.stack(b1s), np.stack(b2s), 1, 16)
    assert t1 == truth and all(found)


def test_size_noisy_pair_falls_back_like_the_oracle(gpu_ctx):
    b1, b2, *_ = make_batch("video_480p", [1], h=120, w=160)
    t1, t2, found = _compare(gpu_ctx, b1, b2, 3, 15, torch.float32)
    assert not found[0] and t1[0] == 15
