"""CUDA path (through the C ABI) against the FP64 oracle on the same inputs.

Tolerances:
  * FP64 path kernels: relative L2 <= 1e-9 (the method's target for the
    double-precision path); f64 latent: relative L2 <= 1e-9.
  * f32 frames deconvolve in single precision: FFT rounding (~1e-6 relative)
    amplified at most 1 / (2 sqrt(eps)) = 50x by the Wiener denominator at
    eps = 1e-4, so latent relative L2 <= 1e-4, and PSNR against the true
    latent within 0.05 dB of the oracle's.
  * Mixed path kernels: relative L2 <= 1e-3; latent PSNR within 0.05 dB.
"""
import numpy as np
import pytest
import torch

import oracle
from tests._inputs import make_batch, psnr, rel

pytestmark = pytest.mark.gpu


def run_gpu(ctx, b1, b2, t1, t2, path, eps, dtype, m=0, flags=0, pad=(0, 0), k1=None, k2=None):
    from paper_1203_4874_gb300 import cbp
    tdt = torch.float64 if dtype == "f64" else torch.float32
    B1 = torch.from_numpy(np.ascontiguousarray(b1)).to(tdt).cuda()
    B2 = torch.from_numpy(np.ascontiguousarray(b2)).to(tdt).cuda()
    flags |= cbp.CBP_FLAG_KERNELS_F64          # compare kernels before any dtype cast
    prm = cbp.params(t1, t2, m=m, path=path, eps=eps, pad_h=pad[0], pad_w=pad[1], flags=flags)
    K1 = None if k1 is None else torch.from_numpy(k1).double().cuda()
    K2 = None if k2 is None else torch.from_numpy(k2).double().cuda()
    lat, k1o, k2o, diag, s = cbp.cbp_deblur_pair(ctx, B1, B2, prm, k1=K1, k2=K2)
    torch.cuda.synchronize()
    return (lat.double().cpu().numpy(), k1o.double().cpu().numpy(), k2o.double().cpu().numpy(),
            [d.as_dict() for d in diag])


def oracle_pair(b1, b2, t1, t2, eps, m=None, **kw):
    return oracle.deblur_pair(b1, b2, t1, t2, m=m, eps=eps, **kw)


def _stage_check(ctx, b1, b2, cfg, path, p_tol, x_tol):
    from paper_1203_4874_gb300 import cbp
    tdt = torch.float64 if cfg.frame_dtype == "f64" else torch.float32
    prm = cbp.params(cfg.t1, cfg.t2, path=path, eps=cfg.eps)
    out = cbp.cbp_estimate_kernels_stages(ctx, torch.from_numpy(b1).to(tdt).cuda(),
                                          torch.from_numpy(b2).to(tdt).cuda(), prm)
    torch.cuda.synchronize()
    o = oracle.estimate_kernels(b1[0], b2[0], cfg.t1, cfg.t2)
    ns = cfg.m // 2 + 1
    for key, okey in (("p_z2", "p_z2_"), ("p_z1", "p_z1_")):
        for k in range(2):
            g = out[key][k][0].cpu().numpy().astype(np.complex128)
            og = o[okey + str(k + 1)][:, :ns]
            assert np.abs(g - og).max() <= p_tol * np.abs(og).max(), (key, k)
    for key in ("x_z2", "x_z1"):
        g = out[key][0].cpu().numpy()
        for s in range(ns):
            ov = abs(np.vdot(g[s], o[key][s])) / (np.linalg.norm(g[s]) * np.linalg.norm(o[key][s]))
            assert 1 - ov <= x_tol, (key, s, 1 - ov)
    sd = out["sample_diag"][0].cpu().numpy()
    sv = np.stack([o["sv_z2"][:ns], o["sv_z1"][:ns]])
    assert np.allclose(sd[..., 0], sv[..., 0] ** 2, rtol=1e-5)           # lambda_max
    assert np.allclose(sd[..., 1], sv[..., -2] ** 2, rtol=1e-3)          # second smallest
    _lifted_check(out["lifted"][0].cpu().numpy(), o, x_tol)
    _diag_check(out["diag"][0], o, 1e-6 if path == "fp64" else 1e-4)
    return out, o


def _phase_free(g, o):
    """1 - |<g, o>| / (|g| |o|) and the norm ratio |g| / |o|."""
    ng, no = np.linalg.norm(g), np.linalg.norm(o)
    return 1 - abs(np.vdot(g, o)) / (ng * no), ng / no


def _lifted_check(lifted, o, tol):
    """A4's lifted spectra against the oracle's a_hat / b_hat.  Each column j of
    A_k (z2-first order) comes from sample j's cofactor vector, each row i of
    B_k (z1-first) from sample i's; a vector's phase is arbitrary, its norm
    (unit cofactors) is not: both kernels' column (row) stacked, compared
    phase-free, with equal norms."""
    a, b = lifted[:2], lifted[2:]
    m = a.shape[1]
    for j in range(m):
        d, r = _phase_free(a[:, :, j].ravel(), o["a_hat"][:, :, j].ravel())
        assert d <= tol and abs(r - 1) <= 1e-6, ("A", j, d, r)
    for i in range(m):
        d, r = _phase_free(b[:, i, :].ravel(), o["b_hat"][:, i, :].ravel())
        assert d <= tol and abs(r - 1) <= 1e-6, ("B", i, d, r)


def _diag_check(dg, o, rtol):
    """Diagnostics against the oracle's: the worst per-sample conditioning
    1 / (sigma_{n-1} / sigma_1) (the device solves samples j <= M/2, the oracle
    all M; conjugate samples share singular values) and the scale system's
    sigma_min / sigma_max, both invariant to the cofactors' phases.  The scale
    residual's bound: rounding of the 2M-square normal matrix (~1e-16 of its
    largest eigenvalue) enters sigma_min^2; on the mixed path the cofactors
    themselves differ from the oracle's by up to ~1e-8, so rtol is wider."""
    od = o["diag"]
    assert abs(dg.kappa_max - od["kappa"]) <= 1e-3 * od["kappa"], (dg.kappa_max, od["kappa"])
    assert abs(dg.gap_min - od["gap_min"]) <= 1e-3 * od["gap_min"], (dg.gap_min, od["gap_min"])
    assert dg.flagged_samples == 0 or od["flagged_samples"] > 0
    sr, osr = dg.scale_resid, od["scale_resid"]
    assert abs(sr * sr - osr * osr) <= 1e-12 + rtol * osr * osr, (sr, osr)


def test_stages_match_oracle_fp64(gpu_ctx):
    """Sample polynomials to 1e-13 and per-sample null vectors to 1e-12 (phase-free)."""
    for name in ("single_64", "video_480p"):
        b1, b2, *_, cfg = make_batch(name, [0], fast=False)
        out, o = _stage_check(gpu_ctx, b1, b2, cfg, "fp64", 1e-13, 1e-12)
        t1 = cfg.t1
        kd = out["kernels"][0].cpu().numpy()
        assert rel(kd[:t1 * t1].reshape(t1, t1), o["k1"]) <= 1e-9


def test_stages_match_oracle_mixed_1080p(gpu_ctx):
    """Mixed path: samples from the exact float fold (1e-12); null vectors after
    one exact-residual step from a single-precision Gram (1e-8)."""
    b1, b2, *_, cfg = make_batch("rgb_1080p", [0])
    _stage_check(gpu_ctx, b1, b2, cfg, "mixed", 1e-12, 1e-8)


def test_full_batch_1080p_as_benchmarked(gpu_ctx):
    """The benchmark's launch configuration (60 pairs of 1080p RGB per call),
    built from two host-generated pairs tiled 30 times; every pair's kernels
    against the oracle (mixed <= 1e-3, FP64 <= 1e-9), latents sampled."""
    from paper_1203_4874_gb300 import cbp
    b1, b2, k1, k2, lat, cfg = make_batch("rgb_1080p", [0, 1])
    refs = [oracle_pair(b1[i], b2[i], 15, 17, cfg.eps) for i in range(2)]
    idx = [i % 2 for i in range(60)]
    B1 = torch.from_numpy(b1).float().cuda()[idx].contiguous()
    B2 = torch.from_numpy(b2).float().cuda()[idx].contiguous()
    for path, tol in (("mixed", 1e-3), ("fp64", 1e-9)):
        prm = cbp.params(15, 17, path=path, eps=cfg.eps, flags=cbp.CBP_FLAG_KERNELS_F64)
        L, K1, K2, diag, _ = cbp.cbp_deblur_pair(gpu_ctx, B1, B2, prm)
        torch.cuda.synchronize()
        K1, K2 = K1.cpu().numpy(), K2.cpu().numpy()
        for f in range(60):
            o = refs[idx[f]]
            assert rel(K1[f], o["k1"]) <= tol and rel(K2[f], o["k2"]) <= tol, (path, f)
        for f in (0, 59):
            g = L[f].double().cpu().numpy()
            o = refs[idx[f]]["latent"]
            assert abs(psnr(g, lat[idx[f]]) - psnr(o, lat[idx[f]])) <= 0.05, (path, f)
            for ch in range(3):
                assert rel(g[ch], o[ch]) <= 1e-4, (path, f, ch, rel(g[ch], o[ch]))
        del L


def test_even_sample_count_self_conjugate_sample(gpu_ctx):
    """M even: sample M/2 is its own conjugate (real polynomials)."""
    rng = np.random.default_rng(13)
    lat = rng.uniform(size=(1, 30, 26))
    from cbp_synth import draw_kernel_pair
    k1, k2 = draw_kernel_pair(rng, 5, 3, 6)
    b1, b2 = oracle.blur_pair(lat, k1, k2)
    g_lat, g_k1, g_k2, diag = run_gpu(gpu_ctx, b1[None], b2[None], 5, 3, "fp64", 0.0, "f64", m=6)
    o = oracle_pair(b1, b2, 5, 3, 0.0, m=6)
    assert rel(g_k1[0], o["k1"]) <= 1e-9 and rel(g_k2[0], o["k2"]) <= 1e-9
    assert rel(g_lat[0], o["latent"]) <= 1e-9


def test_single_64_fp64_exact(gpu_ctx):
    b1, b2, k1, k2, lat, cfg = make_batch("single_64", [0], fast=False)
    g_lat, g_k1, g_k2, diag = run_gpu(gpu_ctx, b1, b2, 5, 5, "fp64", 0.0, "f64")
    o = oracle_pair(b1[0], b2[0], 5, 5, 0.0)
    assert rel(g_k1[0], o["k1"]) <= 1e-9 and rel(g_k2[0], o["k2"]) <= 1e-9
    assert rel(g_k1[0], k1[0]) <= 1e-9 and rel(g_k2[0], k2[0]) <= 1e-9
    assert rel(g_lat[0], o["latent"]) <= 1e-9
    assert diag[0]["status"] == 0
    assert abs(diag[0]["gap_min"] - o["diag"]["gap_min"]) <= 1e-3 * o["diag"]["gap_min"]


def test_video_480p_fp64_batch(gpu_ctx):
    frames = [0, 1, 2]
    b1, b2, k1, k2, lat, cfg = make_batch("video_480p", frames)
    g_lat, g_k1, g_k2, diag = run_gpu(gpu_ctx, b1, b2, 9, 11, "fp64", cfg.eps, "f32")
    for i in range(len(frames)):
        o = oracle_pair(b1[i], b2[i], 9, 11, cfg.eps)
        assert rel(g_k1[i], o["k1"]) <= 1e-9, i
        assert rel(g_k2[i], o["k2"]) <= 1e-9, i
        assert rel(g_lat[i], o["latent"]) <= 1e-4, i
        assert abs(psnr(g_lat[i], lat[i]) - psnr(o["latent"], lat[i])) <= 0.05


def test_rgb_1080p_mixed_and_fp64(gpu_ctx):
    b1, b2, k1, k2, lat, cfg = make_batch("rgb_1080p", [0])
    o = oracle_pair(b1[0], b2[0], 15, 17, cfg.eps)
    g_lat, g_k1, g_k2, diag = run_gpu(gpu_ctx, b1, b2, 15, 17, "mixed", cfg.eps, "f32")
    assert rel(g_k1[0], o["k1"]) <= 1e-3 and rel(g_k2[0], o["k2"]) <= 1e-3
    assert abs(psnr(g_lat[0], lat[0]) - psnr(o["latent"], lat[0])) <= 0.05
    for ch in range(3):
        assert rel(g_lat[0][ch], o["latent"][ch]) <= 1e-4, ch
    f_lat, f_k1, f_k2, _ = run_gpu(gpu_ctx, b1, b2, 15, 17, "fp64", cfg.eps, "f32")
    assert rel(f_k1[0], o["k1"]) <= 1e-9 and rel(f_k2[0], o["k2"]) <= 1e-9
    assert rel(f_lat[0], o["latent"]) <= 1e-4


def test_ragged_sizes_channels_and_extra_samples(gpu_ctx):
    """H, W not multiples of anything, t1 != t2, M > max(t), two channels, f64."""
    rng = np.random.default_rng(11)
    lat = rng.uniform(size=(2, 37, 53))
    from cbp_synth import draw_kernel_pair
    k1, k2 = draw_kernel_pair(rng, 4, 7, 9)
    b1, b2 = oracle.blur_pair(lat, k1, k2)
    g_lat, g_k1, g_k2, diag = run_gpu(gpu_ctx, b1[None], b2[None], 4, 7, "fp64", 0.0, "f64", m=9)
    o = oracle_pair(b1, b2, 4, 7, 0.0, m=9)
    assert rel(g_k1[0], o["k1"]) <= 1e-9 and rel(g_k2[0], o["k2"]) <= 1e-9
    assert rel(g_k1[0], k1) <= 1e-9
    assert rel(g_lat[0], o["latent"]) <= 1e-9


def test_largest_kernels_two_columns_per_lane(gpu_ctx):
    """t1 + t2 = 60 (per-sample systems of 60 unknowns, the scale system 2M = 62):
    the warp-level solvers' lanes each own two columns.  Noise-free f64 frames:
    FP64 path within 1e-9 of the oracle and of the true kernels; mixed path within
    1e-6 of the FP64 path (bar 1e-3)."""
    rng = np.random.default_rng(29)
    lat = rng.uniform(size=(2, 40, 44))
    from cbp_synth import draw_kernel_pair
    k1, k2 = draw_kernel_pair(rng, 29, 31, 31)
    b1, b2 = oracle.blur_pair(lat, k1, k2)
    g_lat, g_k1, g_k2, _ = run_gpu(gpu_ctx, b1[None], b2[None], 29, 31, "fp64", 0.0, "f64")
    o = oracle_pair(b1, b2, 29, 31, 0.0)
    assert rel(g_k1[0], o["k1"]) <= 1e-9 and rel(g_k2[0], o["k2"]) <= 1e-9
    assert rel(g_k1[0], k1) <= 1e-9 and rel(g_k2[0], k2) <= 1e-9
    assert rel(g_lat[0], o["latent"]) <= 1e-9
    _, m_k1, m_k2, _ = run_gpu(gpu_ctx, b1[None], b2[None], 29, 31, "mixed", 0.0, "f64")
    assert rel(m_k1[0], g_k1[0]) <= 1e-6 and rel(m_k2[0], g_k2[0]) <= 1e-6


def test_batch_invariance_and_determinism(gpu_ctx):
    b1, b2, *_ , cfg = make_batch("video_480p", [4, 5, 6], h=96, w=128)
    a_lat, a_k1, a_k2, _ = run_gpu(gpu_ctx, b1, b2, 9, 11, "mixed", cfg.eps, "f32")
    b_lat, b_k1, b_k2, _ = run_gpu(gpu_ctx, b1, b2, 9, 11, "mixed", cfg.eps, "f32")
    assert np.array_equal(a_lat, b_lat) and np.array_equal(a_k1, b_k1)
    for i in range(3):
        s_lat, s_k1, s_k2, _ = run_gpu(gpu_ctx, b1[i:i + 1], b2[i:i + 1], 9, 11, "mixed", cfg.eps, "f32")
        assert np.array_equal(s_lat[0], a_lat[i]) and np.array_equal(s_k2[0], a_k2[i])


def test_strided_frames_match_contiguous(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_ , cfg = make_batch("video_480p", [7], h=64, w=80)
    prm = cbp.params(9, 11, path="fp64", eps=cfg.eps)
    B1 = torch.from_numpy(b1).float().cuda()
    B2 = torch.from_numpy(b2).float().cuda()
    P1 = torch.zeros(B1.shape[:-1] + (B1.shape[-1] + 13,), device="cuda")
    P1[..., :B1.shape[-1]] = B1
    V1 = P1[..., :B1.shape[-1]]
    l0, k0, _, _, _ = cbp.cbp_deblur_pair(gpu_ctx, B1, B2, prm)
    l1, k1, _, _, _ = cbp.cbp_deblur_pair(gpu_ctx, V1, B2, prm)
    torch.cuda.synchronize()
    assert torch.equal(l0, l1) and torch.equal(k0, k1)


def test_known_kernels_single_kernel_and_odd_grid(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, k1, k2, lat, cfg = make_batch("single_64", [1], fast=False)
    eps = 1e-3
    # deconvolution only, true kernels, odd FFT width
    g_lat, *_ = run_gpu(gpu_ctx, b1, b2, 5, 5, "fp64", eps, "f64", flags=cbp.CBP_FLAG_KERNELS_IN,
                        k1=k1, k2=k2, pad=(72, 75))
    o = oracle.deconvolve_dual(b1[0], b2[0], k1[0], k2[0], 64, 64, eps, 72, 75)
    assert rel(g_lat[0], o) <= 1e-9
    # the paper's single-kernel form
    g_lat, *_ = run_gpu(gpu_ctx, b1, b2, 5, 5, "fp64", eps, "f64",
                        flags=cbp.CBP_FLAG_KERNELS_IN | cbp.CBP_FLAG_SINGLE_KERNEL, k1=k1, k2=k2)
    o = oracle.deconvolve_dual(b1[0], b2[0], k1[0], np.zeros_like(k2[0]), 64, 64, eps)
    assert rel(g_lat[0], o) <= 1e-9


def test_host_io_matches_device_path(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_ , cfg = make_batch("video_480p", [8], h=64, w=96)
    prm = cbp.params(9, 11, path="mixed", eps=cfg.eps)
    B1 = torch.from_numpy(b1).float()
    B2 = torch.from_numpy(b2).float()
    ld, kd, _, _, _ = cbp.cbp_deblur_pair(gpu_ctx, B1.cuda(), B2.cuda(), prm)
    prm_h = cbp.params(9, 11, path="mixed", eps=cfg.eps, flags=cbp.CBP_FLAG_HOST_IO)
    lh, kh, _, _, _ = cbp.cbp_deblur_pair(gpu_ctx, B1.pin_memory(), B2.pin_memory(), prm_h)
    torch.cuda.synchronize()
    assert torch.equal(ld.cpu(), lh) and torch.equal(kd.cpu(), kh)


def test_host_io_chunked_pipeline_matches_device_path(gpu_ctx):
    """40 pairs with host I/O: the call splits into five chunks whose inputs go over in
    order on one copy stream while earlier chunks compute (three compute streams);
    every pair's latent and kernels equal the device-resident call's."""
    from paper_1203_4874_gb300 import cbp
    b1, b2, *_, cfg = make_batch("video_480p", [8, 9, 10, 11, 12], h=64, w=96)
    idx = [(7 * i) % 5 for i in range(40)]
    B1 = torch.from_numpy(b1).float()[idx].contiguous()
    B2 = torch.from_numpy(b2).float()[idx].contiguous()
    prm = cbp.params(9, 11, path="mixed", eps=cfg.eps)
    ld, kd, kd2, _, _ = cbp.cbp_deblur_pair(gpu_ctx, B1.cuda(), B2.cuda(), prm)
    prm_h = cbp.params(9, 11, path="mixed", eps=cfg.eps, flags=cbp.CBP_FLAG_HOST_IO)
    lh, kh, kh2, _, _ = cbp.cbp_deblur_pair(gpu_ctx, B1.pin_memory(), B2.pin_memory(), prm_h)
    torch.cuda.synchronize()
    assert torch.equal(ld.cpu(), lh) and torch.equal(kd.cpu(), kh) and torch.equal(kd2.cpu(), kh2)


def test_non_finite_input_is_reported(gpu_ctx):
    b1, b2, *_ = make_batch("single_64", [2], fast=False)
    b1 = b1.copy()
    b1[0, 0, 10, 10] = np.nan
    *_, diag = run_gpu(gpu_ctx, b1, b2, 5, 5, "fp64", 0.0, "f64")
    assert diag[0]["status"] == -1


def test_forward_model_matches_oracle(gpu_ctx):
    from paper_1203_4874_gb300 import cbp
    rng = np.random.default_rng(12)
    lat = rng.uniform(size=(2, 1, 33, 45))
    ks = np.stack([rng.uniform(size=(6, 6)) for _ in range(2)])
    out = cbp.cbp_forward_blur(gpu_ctx, torch.from_numpy(lat).cuda(), torch.from_numpy(ks).cuda())
    torch.cuda.synchronize()
    for i in range(2):
        assert rel(out[i, 0].cpu().numpy(), oracle.blur_full(lat[i, 0], ks[i])) <= 1e-14
    # float frames: Eq. 1 accumulated in float32 (the precision they are stored in)
    lat32 = lat.astype(np.float32)
    ks15 = np.stack([rng.uniform(size=(15, 15)) for _ in range(2)])
    out32 = cbp.cbp_forward_blur(gpu_ctx, torch.from_numpy(lat32).cuda(), torch.from_numpy(ks15).cuda())
    torch.cuda.synchronize()
    for i in range(2):
        ref = oracle.blur_full(lat32[i, 0].astype(np.float64), ks15[i])
        # float taps and a float sum of t^2 = 225 positive terms: at most about
        # (t^2 + 1) u = 1.3e-5 relative, typically ~2e-7
        assert rel(out32[i, 0].double().cpu().numpy(), ref) <= 2e-6
    # noise: sample mean and variance of sigma * N(0, 1) on a zero latent
    z = torch.zeros((1, 1, 400, 400), dtype=torch.float32, device="cuda")
    delta = torch.zeros((1, 1, 1), dtype=torch.float64, device="cuda")
    nz = cbp.cbp_forward_blur(gpu_ctx, z, delta, sigma=1e-3, seed=5).double().cpu().numpy()
    assert abs(nz.mean()) < 2e-5 and abs(nz.std() / 1e-3 - 1) < 1e-2


def test_mixed_path_near_degenerate_samples(gpu_ctx):
    """1080p pairs from the device forward model whose z = 1 samples have their
    two smallest eigenvalues ~1e-8 lambda_max apart (pair 4 of this seed): the
    mixed path's kernels stay within 1e-3 of the FP64 path's (measured ~1e-8)."""
    import bench
    from paper_1203_4874_gb300 import cbp
    dev = torch.device("cuda", 0)
    b1, b2, _, _ = bench.make_inputs(gpu_ctx, 5, 1203000, dev)
    out = {}
    for path in ("mixed", "fp64"):
        prm = cbp.params(15, 17, path=path, eps=1e-4, flags=cbp.CBP_FLAG_KERNELS_F64)
        k1, k2, _, _ = cbp.cbp_estimate_kernels(gpu_ctx, b1, b2, prm)
        out[path] = torch.cat([k1.flatten(1), k2.flatten(1)], dim=1)
    torch.cuda.synchronize()
    err = ((out["mixed"] - out["fp64"]).norm(dim=1) / out["fp64"].norm(dim=1)).max().item()
    assert err <= 1e-3, err
