"""Pins of the camera-side oracle (Section 3: random kernels drawn anew for
every frame, kept when coprime; the cascaded pair): Philox-4x32-10 against
its published known-answer vectors, the kernel draw's normalisation and
independence, the coprimality test against planted shared roots, a two-tap
closed form and the exact resultant, and Eq. 4's identity for the direct and
the cascaded pairs."""
import numpy as np
import pytest
from scipy.signal import convolve2d

import oracle
from oracle import camera


def test_philox_known_answers():
    # Random123's known-answer vectors for Philox-4x32 with 10 rounds
    kat = [((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
           ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
           ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
            (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for ctr, key, want in kat:
        assert camera.philox4x32_10(ctr, key) == want


def test_kernel_draw_normalised_positive_and_independent():
    k = camera.draw_kernel(99, 3, 0, 0, 15)
    assert k.shape == (15, 15) and np.all(k > 0) and abs(k.sum() - 1.0) <= 1e-15
    assert np.array_equal(k, camera.draw_kernel(99, 3, 0, 0, 15))
    others = [camera.draw_kernel(99, 4, 0, 0, 15), camera.draw_kernel(99, 3, 1, 0, 15),
              camera.draw_kernel(99, 3, 0, 1, 15), camera.draw_kernel(98, 3, 0, 0, 15)]
    for o in others:
        assert not np.allclose(k, o)
    # the raw uniforms: entry e is word e mod 4 of block e // 4, (word + 1) 2^-32
    u = [(camera.philox4x32_10((e // 4, 3, 0, 0), (99, 0))[e % 4] + 1.0) * 2.0 ** -32
         for e in range(225)]
    total = 0.0
    for v in u:
        total += v
    assert np.array_equal(k.ravel(), np.array(u) / total)


def test_two_tap_closed_form():
    """Linear factors a0 + a1 z and b0 + b1 z share a root iff a0 b1 = a1 b0."""
    k1 = np.array([[1.0, 2.0], [3.0, 4.0]])
    k2 = np.array([[2.0, 4.0], [1.0, 5.0]])
    r = camera.coprime_ratios(k1, k2, 2)
    # order 0, sample j: a = k1 @ w, a_j = (k1[0] . w_j, k1[1] . w_j); closed form singularity
    w = oracle.root_powers(2, 2)
    for j in range(2):
        a, b = k1 @ w[:, j], k2 @ w[:, j]
        shared = abs(a[0] * b[1] - a[1] * b[0]) < 1e-12
        assert (r[j][0] < 1e-12) == shared
    # planted: equal row sums (3, 7) make the z2 = 1 sample share its root
    k2 = np.array([[1.5, 1.5], [3.5, 3.5]])
    r = camera.coprime_ratios(k1, k2, 2)
    assert r[0][0] < 1e-12 and not camera.is_coprime(k1, k2, 2)   # order 0, sample 0


def test_planted_shared_factor_fails_and_random_pairs_pass():
    rng = np.random.default_rng(4)
    a1, a2 = rng.uniform(size=(4, 4)), rng.uniform(size=(5, 5))
    g = np.array([[1.0, 0.3], [0.2, 0.9]])
    assert not camera.is_coprime(convolve2d(a1, g), convolve2d(a2, g), 6)
    ratios = camera.coprime_ratios(convolve2d(a1, g), convolve2d(a2, g), 6)
    assert all(r <= 1e-12 for r, _ in ratios)
    for f in range(5):
        k1, k2, att = camera.draw_pair(7, f, 5, 5, 5)
        assert att >= 0 and camera.is_coprime(k1, k2, 5)
        assert oracle.resultant_nonzero(k1, k2)


def test_eq4_identity_for_the_pair_and_the_cascade():
    rng = np.random.default_rng(8)
    lat = rng.uniform(size=(1, 20, 23))
    out = camera.encrypt(lat, 11, 0, 5, 4, cascade=(3, 5))
    b1, b2, c1, c2 = out["b1"][0], out["b2"][0], out["c1"][0], out["c2"][0]
    lhs, rhs = convolve2d(b1, out["k2"]), convolve2d(b2, out["k1"])
    assert np.max(np.abs(lhs - rhs)) <= 1e-14 * np.max(np.abs(lhs))
    lhs, rhs = convolve2d(c1, out["k4"]), convolve2d(c2, out["k3"])
    assert np.max(np.abs(lhs - rhs)) <= 1e-14 * np.max(np.abs(lhs))
    assert np.allclose(c1, convolve2d(b1, out["k3"]), rtol=0, atol=1e-15)
