"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
closed forms, brute force, exact rational arithmetic, a library routine, or
the paper's identities (Eq. 1-4).  The mutation tests at the end plant a
plausible mistake in the oracle and show that a pin catches it.
"""
import cmath
import math

import numpy as np
import pytest
import scipy.signal

import oracle
from cbp_synth import CONFIGS, draw_kernel_pair, make_pair_inputs, uniform_kernel

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def brute_poly_eval(coeffs, z):
    """Horner's rule, lowest degree first."""
    acc = 0j
    for c in reversed(list(coeffs)):
        acc = acc * z + c
    return acc


# --------------------------------------------------------------- Eq. 1 ------
def test_blur_shifted_delta_is_a_shift():
    rng = np.random.default_rng(1)
    lat = rng.uniform(size=(7, 9))
    k = np.zeros((4, 4))
    k[2, 1] = 1.0
    b = oracle.blur_full(lat, k)
    expect = np.zeros((10, 12))
    expect[2:9, 1:10] = lat
    assert np.array_equal(b, expect)


def test_blur_matches_library_full_convolution():
    rng = np.random.default_rng(2)
    lat = rng.uniform(size=(11, 8))
    k = rng.uniform(size=(5, 5))          # asymmetric: a flipped kernel would fail
    assert rel(oracle.blur_full(lat, k), scipy.signal.convolve2d(lat, k, mode="full")) < 1e-14


def test_coprime_pair_identity_eq4():
    """b1 k2 = l k1 k2 = b2 k1 (Eq. 4), outer products by a library convolution."""
    inp = make_pair_inputs("single_64")
    b1, b2 = oracle.blur_pair(inp.latent, inp.k1, inp.k2)
    lhs = scipy.signal.convolve2d(b1[0], inp.k2)
    rhs = scipy.signal.convolve2d(b2[0], inp.k1)
    assert rel(lhs, rhs) < 1e-14


# ------------------------------------------------------------ Eq. 2-3 -------
def test_evaluation_is_polynomial_evaluation():
    rng = np.random.default_rng(3)
    b = rng.standard_normal((1, 5, 6))
    m = 5
    pz2 = oracle.evaluate_z2(b, m)
    pz1 = oracle.evaluate_z1(b, m)
    for j in range(m):
        w = cmath.exp(-2j * math.pi * j / m)
        for r in range(5):
            assert abs(pz2[0, j, r] - brute_poly_eval(b[0, r, :], w)) < 1e-13
        for c in range(6):
            assert abs(pz1[0, j, c] - brute_poly_eval(b[0, :, c], w)) < 1e-13
    assert np.allclose(pz2[0, 0].real, b[0].sum(axis=1), atol=1e-13)
    assert np.allclose(pz1[0, 0].real, b[0].sum(axis=0), atol=1e-13)
    # Eq. 3: b(z1, z2) = z1^T B z2 from either order
    for i in range(m):
        for j in range(m):
            zi, zj = cmath.exp(-2j * math.pi * i / m), cmath.exp(-2j * math.pi * j / m)
            direct = sum(b[0, r, c] * zi ** r * zj ** c for r in range(5) for c in range(6))
            assert abs(brute_poly_eval(pz2[0, j], zi) - direct) < 1e-12
            assert abs(brute_poly_eval(pz1[0, i], zj) - direct) < 1e-12


def test_convolution_and_sylvester_matrices():
    rng = np.random.default_rng(4)
    b1 = rng.standard_normal(9) + 1j * rng.standard_normal(9)    # H + t1 - 1, H = 5
    b2 = rng.standard_normal(7) + 1j * rng.standard_normal(7)    # H + t2 - 1
    u = rng.standard_normal(5) + 1j * rng.standard_normal(5)   # t1 = 5
    v = rng.standard_normal(3) + 1j * rng.standard_normal(3)   # t2 = 3
    assert np.allclose(oracle.convolution_matrix(b1, 3) @ v, np.convolve(b1, v), atol=1e-13)
    s = oracle.sylvester_system([b1], [b2], 5, 3)
    assert np.allclose(s @ np.concatenate([u, v]), np.convolve(b1, v) - np.convolve(b2, u), atol=1e-13)


# ------------------------------------------------------- Eq. 4, Section 4 ---
def _true_cofactors(k1, k2, m, axis):
    """[k1(., w^s); k2(., w^s)] by direct sums (axis 1: z2 substituted)."""
    out = []
    for s in range(m):
        w = cmath.exp(-2j * math.pi * s / m)
        vec = []
        for k in (k1, k2):
            t = k.shape[0]
            for p in range(t):
                if axis == 1:
                    vec.append(sum(k[p, q] * w ** q for q in range(t)))
                else:
                    vec.append(sum(k[q, p] * w ** q for q in range(t)))
        out.append(np.array(vec))
    return out


def test_null_vectors_are_the_true_cofactors_noise_free():
    inp = make_pair_inputs("single_64")
    b1, b2 = oracle.blur_pair(inp.latent, inp.k1, inp.k2)
    out = oracle.estimate_kernels(b1, b2, 5, 5)
    for key, axis in (("x_z2", 1), ("x_z1", 0)):
        for s, xt in enumerate(_true_cofactors(inp.k1, inp.k2, 5, axis)):
            ov = abs(np.vdot(out[key][s], xt)) / np.linalg.norm(xt)
            assert ov >= 1 - 1e-12, (key, s, ov)


def test_exact_recovery_single_64():
    """Noise-free 64x64 pair, 5x5 kernels, eps = 0: kernels and latent exact."""
    cfg = CONFIGS["single_64"]
    inp = make_pair_inputs(cfg)
    b1, b2 = oracle.blur_pair(inp.latent, inp.k1, inp.k2)
    out = oracle.deblur_pair(b1, b2, 5, 5, eps=0.0)
    assert rel(out["k1"], inp.k1) < 1e-10
    assert rel(out["k2"], inp.k2) < 1e-10
    assert rel(out["latent"], inp.latent) < 1e-10
    kappa = out["diag"]["kappa"]
    assert rel(out["k1"], inp.k1) < 1e-14 * kappa * 100


def test_resultant_certifies_generated_pair_and_rejects_common_factor():
    inp = make_pair_inputs("single_64")
    assert oracle.resultant_nonzero(inp.k1, inp.k2)
    # small integers keep the planted common factor exact in floating point
    rng = np.random.default_rng(5)
    g = rng.integers(1, 9, size=(2, 2)).astype(float)
    a = rng.integers(1, 9, size=(3, 3)).astype(float)
    c = rng.integers(1, 9, size=(3, 3)).astype(float)
    assert oracle.resultant_nonzero(a, c)
    assert not oracle.resultant_nonzero(scipy.signal.convolve2d(a, g), scipy.signal.convolve2d(c, g))
    # a common factor in z2 only still leaves Res_z1 non-zero; Res_z2 catches it
    gz2 = np.array([[2.0, 1.0]])      # 2 + z2
    a4 = rng.integers(1, 9, size=(4, 3)).astype(float)
    c4 = rng.integers(1, 9, size=(4, 3)).astype(float)
    k1 = scipy.signal.convolve2d(a4, gz2)
    k2 = scipy.signal.convolve2d(c4, gz2)
    assert not oracle.resultant_nonzero(k1, k2)


def test_separable_kernels_closed_form():
    """K_k = a_k b_k^T: cofactors are b_k(w^j) a_k, spectra rank one, LS residual 0."""
    rng = np.random.default_rng(6)
    a1, b1v = np.array([1.0, 0.5, 0.2]), np.array([1.0, -0.3, 0.6])
    a2, b2v = np.array([1.0, 0.9, 0.1, 0.3]), np.array([0.7, 0.2, 1.0, 0.4])
    s1, s2 = a1.sum() * b1v.sum(), a2.sum() * b2v.sum()
    k1 = np.outer(a1, b1v) / s1
    k2 = np.outer(a2, b2v) / s2
    lat = rng.uniform(size=(1, 20, 18))
    bb1, bb2 = oracle.blur_pair(lat, k1, k2)
    m = 4
    out = oracle.estimate_kernels(bb1, bb2, 3, 4, m)
    for s in range(m):
        w = cmath.exp(-2j * math.pi * s / m)
        xt = np.concatenate([brute_poly_eval(b1v, w) * a1 / s1, brute_poly_eval(b2v, w) * a2 / s2])
        assert abs(np.vdot(out["x_z2"][s], xt)) / np.linalg.norm(xt) > 1 - 1e-12
    for k in range(2):
        sv = np.linalg.svd(out["x_k"][k], compute_uv=False)
        assert sv[1] / sv[0] < 1e-12
    assert out["diag"]["scale_resid"] < 1e-12
    assert rel(out["k1"], k1) < 1e-10 and rel(out["k2"], k2) < 1e-10


def test_scale_least_squares_inverts_per_sample_scales():
    rng = np.random.default_rng(7)
    m = 5
    ks = [uniform_kernel(rng, 4), uniform_kernel(rng, 5)]
    kh = [np.fft.fft2(k, s=(m, m)) for k in ks]       # library DFT of the true kernels
    c = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    d = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    a = np.stack([c[None, :] * x for x in kh])
    b = np.stack([d[:, None] * x for x in kh])
    gamma, delta, sv = oracle.scale_least_squares(a, b)
    g = gamma * c
    assert np.allclose(g, g[0], rtol=1e-12, atol=0)
    assert np.allclose(delta * d, g[0], rtol=1e-12, atol=0)
    assert sv[-1] / sv[0] < 1e-13
    xk = oracle.kernel_spectra(a, b, gamma, delta)
    for k in range(2):
        assert np.allclose(xk[k], kh[k] / kh[k][0, 0], atol=1e-12)


def test_inverse_dft_of_kernel_spectrum():
    rng = np.random.default_rng(8)
    k = rng.uniform(size=(4, 4))
    x = np.fft.fft2(k, s=(6, 6))
    kk, full = oracle.kernels_from_spectra(x, 4)
    assert np.allclose(kk, k, atol=1e-13)
    assert np.allclose(full, np.fft.ifft2(x), atol=1e-13)


# ---------------------------------------------------------- deconvolution ---
def test_dual_deconvolution_with_shifted_deltas_closed_form():
    """K_k = delta(p_k, q_k): I^ = 2 L^ / (2 + eps), so latent = 2 L / (2 + eps)."""
    rng = np.random.default_rng(9)
    lat = rng.uniform(size=(2, 9, 11))
    k1 = np.zeros((3, 3)); k1[1, 2] = 1.0
    k2 = np.zeros((4, 4)); k2[3, 0] = 1.0
    b1, b2 = oracle.blur_pair(lat, k1, k2)
    eps = 0.3
    out = oracle.deconvolve_dual(b1, b2, k1, k2, 9, 11, eps)
    assert np.allclose(out, 2.0 * lat / (2.0 + eps), atol=1e-13)


def _direct_dft2(x, ph, pw, sign):
    out = np.zeros((ph, pw), complex)
    for u in range(ph):
        for v in range(pw):
            acc = 0j
            for r in range(x.shape[0]):
                for c in range(x.shape[1]):
                    acc += x[r, c] * cmath.exp(sign * 2j * math.pi * (u * r / ph + v * c / pw))
            out[u, v] = acc
    return out


def test_single_kernel_form_is_textbook_wiener_by_direct_dft():
    """K2 = 0 reduces the dual formula to conj(K^) B^ / (|K^|^2 + eps); spectra by brute force."""
    rng = np.random.default_rng(10)
    lat = rng.uniform(size=(1, 4, 5))
    k1 = rng.uniform(size=(2, 2))
    k2 = np.zeros((3, 3))
    b1, b2 = oracle.blur_pair(lat, k1, k2)
    ph, pw = 6, 7
    eps = 0.05
    got = oracle.deconvolve_dual(b1, b2, k1, k2, 4, 5, eps, ph, pw)
    fb = _direct_dft2(b1[0], ph, pw, -1)
    fk = _direct_dft2(k1, ph, pw, -1)
    ih = np.conj(fk) * fb / (np.abs(fk) ** 2 + eps)
    lat_hat = _direct_dft2(ih, ph, pw, +1).real / (ph * pw)
    assert np.allclose(got[0], lat_hat[:4, :5], atol=1e-12)


def test_fft_grid_size_is_smallest_7_smooth():
    smooth = [k for k in range(1, 3000) if all(p in (2, 3, 5, 7) for p in _factors(k))]
    for n in range(1, 2000, 7):
        assert oracle.fft_grid_size(n) == min(s for s in smooth if s >= n)
    assert oracle.fft_grid_size(1096) == 1120 and oracle.fft_grid_size(1936) == 1944


def _factors(k):
    out, d = [], 2
    while d * d <= k:
        while k % d == 0:
            out.append(d)
            k //= d
        d += 1
    if k > 1:
        out.append(k)
    return out


# ------------------------------------------------------------- generators ---
def test_generators_are_seeded_and_normalised():
    a = make_pair_inputs("video_480p", 3, h=48, w=64)
    b = make_pair_inputs("video_480p", 3, h=48, w=64)
    assert np.array_equal(a.latent, b.latent) and np.array_equal(a.noise1, b.noise1)
    assert abs(a.k1.sum() - 1) < 1e-14 and abs(a.k2.sum() - 1) < 1e-14
    assert a.k1.shape == (9, 9) and a.k2.shape == (11, 11)
    k1, k2 = draw_kernel_pair(11, 15, 17, 17, "mixture")
    assert abs(k1.sum() - 1) < 1e-14 and (k1 >= 0).all()


# --------------------------------------------------------------- mutations --
def test_pins_catch_planted_mistakes(monkeypatch):
    """A flipped root sign, a missing conjugate or a wrong Sylvester sign each
    break a pin above."""
    import oracle.cbp_oracle as oc

    orig_root = oc.root_powers
    monkeypatch.setattr(oc, "root_powers", lambda n, m, sign=-1: orig_root(n, m, -sign))
    with pytest.raises(AssertionError):
        test_evaluation_is_polynomial_evaluation()
    monkeypatch.setattr(oc, "root_powers", orig_root)

    orig_syl = oc.sylvester_system

    def bad_sylvester(b1s, b2s, t1, t2):
        return np.vstack([np.hstack([oc.convolution_matrix(b2, t1), oc.convolution_matrix(b1, t2)])
                          for b1, b2 in zip(b1s, b2s)])
    monkeypatch.setattr(oc, "sylvester_system", bad_sylvester)
    monkeypatch.setattr(oracle, "sylvester_system", bad_sylvester)
    with pytest.raises(AssertionError):
        test_convolution_and_sylvester_matrices()
    with pytest.raises(AssertionError):       # the cofactors change too
        test_null_vectors_are_the_true_cofactors_noise_free()
    monkeypatch.setattr(oc, "sylvester_system", orig_syl)
    monkeypatch.setattr(oracle, "sylvester_system", orig_syl)

    orig_conj = oc.np.conj
    monkeypatch.setattr(oc.np, "conj", lambda x: x)
    try:
        with pytest.raises(AssertionError):
            test_dual_deconvolution_with_shifted_deltas_closed_form()
    finally:
        monkeypatch.setattr(oc.np, "conj", orig_conj)
