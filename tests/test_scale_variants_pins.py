"""Pins of the oracle's scale-fix variants: the single-pass support-
constrained fix (with M > t the estimate's inverse DFT must vanish outside
the kernel) and the paper's k1-only pipeline (kernel 1's scale equations,
B1 divided by K1, Section 4).  Checked against what the mathematics fixes:
inverting planted per-sample scales, exact recovery on a noise-free pair,
agreement of the k1-only scale with the two-kernel one on exact data, and
the support constraint's need for M > t."""
import numpy as np
import pytest

import oracle
from tests._inputs import make_batch


def _true_lift(k1, k2, m):
    """A_k[i][j] = K_k^[i][j] on the M x M grid (the exact z2-first lift)."""
    a = np.stack([np.fft.fft2(k, s=(m, m)) for k in (k1, k2)])
    return a


def test_support_fix_inverts_planted_scales():
    rng = np.random.default_rng(2)
    k1, k2 = rng.uniform(size=(4, 4)), rng.uniform(size=(5, 5))
    m = 8
    a = _true_lift(k1, k2, m)
    c = rng.normal(size=m) + 1j * rng.normal(size=m)
    gamma, sv = oracle.scale_support(a * c[None, None, :], 4, 5)
    r = gamma * c
    assert np.allclose(r / r[0], np.ones(m), atol=1e-12)
    assert sv[-1] / sv[0] < 1e-13
    x = oracle.kernel_spectra_support(a * c[None, None, :], gamma)
    k1r, _ = oracle.kernels_from_spectra(x[0], 4)
    assert np.allclose(k1r, k1 / k1.sum(), atol=1e-13)


def test_support_fix_needs_more_samples_than_the_kernel():
    rng = np.random.default_rng(3)
    a = _true_lift(rng.uniform(size=(5, 5)), rng.uniform(size=(5, 5)), 5)
    with pytest.raises(ValueError):
        oracle.scale_support(a, 5, 5)


@pytest.mark.parametrize("scale,m", [("support", 7), ("k1", 5)])
def test_exact_recovery_noise_free(scale, m):
    b1, b2, k1, k2, lat, cfg = make_batch("single_64", [0], fast=False)
    o = oracle.deblur_pair(b1[0], b2[0], 5, 5, m=m, eps=0.0, scale=scale)
    assert np.linalg.norm(o["k1"] - k1[0]) <= 1e-10 * np.linalg.norm(k1[0])
    assert np.linalg.norm(o["latent"] - lat[0]) <= 1e-10 * np.linalg.norm(lat[0])
    if scale == "support":
        assert np.linalg.norm(o["k2"] - k2[0]) <= 1e-10 * np.linalg.norm(k2[0])


def test_k1_only_scale_matches_the_two_kernel_scale_on_exact_data():
    b1, b2, *_ = make_batch("single_64", [1], fast=False)
    full = oracle.estimate_kernels(b1[0], b2[0], 5, 5)
    only = oracle.estimate_kernels(b1[0], b2[0], 5, 5, scale="k1")
    g = np.concatenate([full["gamma"], full["delta"]])
    h = np.concatenate([only["gamma"], only["delta"]])
    assert 1 - abs(np.vdot(g, h)) / (np.linalg.norm(g) * np.linalg.norm(h)) <= 1e-12
    assert only["k2"] is None
