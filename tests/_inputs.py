"""Test-input assembly: seeded generators + Eq. 1 applied on the host.

Small cases use the oracle's direct convolution; full-size frames use a
library FFT convolution for speed (inputs only -- the oracle and the CUDA path
then consume the very same arrays).  Frames of f32 workloads are rounded to
float32 first, and the oracle receives the rounded values.
"""
from __future__ import annotations

import numpy as np
import scipy.signal

import oracle
from cbp_synth import CONFIGS, make_pair_inputs


def blur(lat, k, fast):
    if fast:
        return np.stack([scipy.signal.fftconvolve(ch, k, mode="full") for ch in lat])
    return np.stack([oracle.blur_full(ch, k) for ch in lat])


def make_batch(cfg_name, frames, h=None, w=None, fast=None, noise=True):
    cfg = CONFIGS[cfg_name]
    b1s, b2s, k1s, k2s, lats = [], [], [], [], []
    for f in frames:
        inp = make_pair_inputs(cfg, f, h=h, w=w)
        big = (h or cfg.h) * (w or cfg.w) > 300_000
        use_fast = big if fast is None else fast
        b1 = blur(inp.latent, inp.k1, use_fast) + (inp.noise1 if noise else 0)
        b2 = blur(inp.latent, inp.k2, use_fast) + (inp.noise2 if noise else 0)
        if cfg.frame_dtype == "f32":
            b1 = b1.astype(np.float32).astype(np.float64)
            b2 = b2.astype(np.float32).astype(np.float64)
        b1s.append(b1)
        b2s.append(b2)
        k1s.append(inp.k1)
        k2s.append(inp.k2)
        lats.append(inp.latent)
    return (np.stack(b1s), np.stack(b2s), np.stack(k1s), np.stack(k2s), np.stack(lats), cfg)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def psnr(x, ref):
    mse = float(np.mean((np.asarray(x) - np.asarray(ref)) ** 2))
    peak = float(np.max(np.abs(ref)))
    return 10.0 * np.log10(peak * peak / mse) if mse > 0 else float("inf")
