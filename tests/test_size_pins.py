"""Pins of the oracle's kernel-size estimation (Section 4: the kernel degree
from the singularity of the cofactor system; Section 5: a scan of square
candidate sizes with a fallback to the largest).  Checked against what the
mathematics fixes, not against the oracle itself: exact recovery on
noise-free pairs, the null-space dimension t' - t + 1 of the Sylvester
system above the true size (the cofactors times any polynomial of degree
t' - t), full rank below it, and a planted common factor that moves the
detected size."""
import numpy as np
import pytest

import oracle
from cbp_synth import draw_kernel_pair


def _pair(t1, t2, seed, h=36, w=40):
    rng = np.random.default_rng(seed)
    lat = rng.uniform(size=(1, h, w))
    k1, k2 = draw_kernel_pair(rng, t1, t2, max(t1, t2))
    b1, b2 = oracle.blur_pair(lat, k1, k2)
    return b1, b2, k1, k2


@pytest.mark.parametrize("t", [5, 7, 9, 11, 13, 15, 17, 19, 21, 23, 25])
def test_true_size_recovered_noise_free(t):
    b1, b2, *_ = _pair(t, t, 100 + t)
    t1, t2, found, ratios = oracle.estimate_size(b1, b2, 1, t + 2)
    assert (t1, t2, found) == (t, t, True)
    # full rank below the true size, singular from it on
    assert all(ratios[s] > 1e-8 for s in ratios if s < t)
    assert all(ratios[s] < 1e-12 for s in ratios if s >= t)


@pytest.mark.parametrize("t1,t2", [(9, 11), (15, 17), (7, 4)])
def test_unequal_sizes_follow_the_blurred_sizes(t1, t2):
    b1, b2, *_ = _pair(t1, t2, 7 * t1 + t2)
    assert oracle.estimate_size(b1, b2, 1, 20)[:3] == (t1, t2, True)


def test_null_space_dimension_above_the_true_size():
    """At t' >= t the system's null vectors are (k1 s, k2 s), deg s <= t' - t:
    exactly t' - t + 1 singular values vanish, in both evaluation orders."""
    t = 6
    b1, b2, *_ = _pair(t, t, 31)
    r1, c1 = oracle.plane_sums(b1)
    r2, c2 = oracle.plane_sums(b2)
    for tp in range(t, t + 4):
        for p1, p2 in ((r1, r2), (c1, c2)):
            sv = np.linalg.svd(oracle.sylvester_system(p1, p2, tp, tp), compute_uv=False)
            assert int(np.sum(sv <= 1e-11 * sv[0])) == tp - t + 1


def test_plane_sums_are_the_z1_samples():
    rng = np.random.default_rng(3)
    b = rng.normal(size=(2, 7, 9))
    rs, cs = oracle.plane_sums(b)
    assert np.allclose(rs, oracle.evaluate_z2(b, 1)[:, 0, :].real, rtol=0, atol=1e-13)
    assert np.allclose(cs, oracle.evaluate_z1(b, 1)[:, 0, :].real, rtol=0, atol=1e-13)


def test_planted_common_factor_moves_the_detected_size():
    """Kernels sharing a factor are not coprime: the system is singular one
    size early (the cofactors of the shared factor), so a wrong coprimality
    assumption shows."""
    rng = np.random.default_rng(5)
    lat = rng.uniform(size=(1, 30, 34))
    a1, a2 = draw_kernel_pair(rng, 5, 5, 5)
    c = np.array([[1.0, 0.5], [0.25, 0.7]])
    from scipy.signal import convolve2d
    k1, k2 = convolve2d(a1, c), convolve2d(a2, c)
    b1, b2 = oracle.blur_pair(lat, k1, k2)
    t1, t2, found, _ = oracle.estimate_size(b1, b2, 1, 8)
    assert found and (t1, t2) == (5, 5)


def test_noise_without_a_singular_candidate_falls_back_to_the_largest():
    b1, b2, *_ = _pair(7, 7, 9)
    rng = np.random.default_rng(10)
    b1 = b1 + 1e-2 * rng.normal(size=b1.shape)
    b2 = b2 + 1e-2 * rng.normal(size=b2.shape)
    t1, t2, found, ratios = oracle.estimate_size(b1, b2, 1, 11)
    assert not found and (t1, t2) == (11, 11) and min(ratios.values()) > 1e-6
