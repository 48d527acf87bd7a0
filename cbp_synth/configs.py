"""The five CBP workloads as seeded recipes.

Sizes follow the workload definitions: latent H x W, kernels t1 x t1 and
t2 x t2, blurred frames (H + t_k - 1) x (W + t_k - 1) under full convolution.
``make_pair_inputs`` returns everything a frame pair needs *before* the blur:
the latent, both kernels and both noise fields.  Applying Eq. 1 is left to the
caller (the oracle in tests, the library's forward-model kernel in benches).

Seeds:
  single_64    seed 1203 (latent, then kernels drawn from the same stream)
  video_480p   frame f: latent/noise seed 4874 + f; kernels from seed 4874
               (fixed for the whole video)
  rgb_1080p    frame f: seed 1203000 + f for latent, kernels and noise
               (new kernels for every frame, as in Section 3)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .generators import (_rng, blob_latent, draw_kernel_pair, gaussian_noise)


@dataclass(frozen=True)
class Config:
    name: str
    h: int
    w: int
    channels: int
    t1: int
    t2: int
    frames: int
    family: str          # kernel family
    noise_sigma: float
    frame_dtype: str     # "f64" or "f32"
    path: str            # "fp64" or "mixed"
    eps: float           # Wiener regulariser of the dual-kernel deconvolution

    @property
    def m(self) -> int:
        return max(self.t1, self.t2)


CONFIGS = {
    "single_64": Config("single_64", 64, 64, 1, 5, 5, 1, "uniform", 0.0, "f64", "fp64", 0.0),
    "video_480p": Config("video_480p", 480, 640, 1, 9, 11, 30, "uniform", 1e-3, "f32", "fp64", 1e-4),
    "rgb_1080p": Config("rgb_1080p", 1080, 1920, 3, 15, 17, 60, "mixture", 1e-3, "f32", "mixed", 1e-4),
}


@dataclass
class PairInputs:
    latent: np.ndarray      # (C, H, W) float64
    k1: np.ndarray          # (t1, t1)
    k2: np.ndarray          # (t2, t2)
    noise1: np.ndarray      # (C, H + t1 - 1, W + t1 - 1)
    noise2: np.ndarray      # (C, H + t2 - 1, W + t2 - 1)


def make_pair_inputs(cfg: Config | str, frame: int = 0, *, h: int | None = None,
                     w: int | None = None) -> PairInputs:
    """Seeded inputs of one frame pair of ``cfg`` (optionally at a smaller H x W)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    h = cfg.h if h is None else h
    w = cfg.w if w is None else w
    c, t1, t2 = cfg.channels, cfg.t1, cfg.t2
    if cfg.name == "single_64":
        rng = _rng(1203 + frame)
        lat = blob_latent(rng, h, w, c)
        k1, k2 = draw_kernel_pair(rng, t1, t2, cfg.m, cfg.family)
    elif cfg.name == "video_480p":
        rng = _rng(4874 + frame)
        lat = blob_latent(rng, h, w, c)
        k1, k2 = draw_kernel_pair(_rng(4874), t1, t2, cfg.m, cfg.family)
    else:
        rng = _rng(1203000 + frame)
        lat = blob_latent(rng, h, w, c)
        k1, k2 = draw_kernel_pair(rng, t1, t2, cfg.m, cfg.family)
    n1 = gaussian_noise(rng, (c, h + t1 - 1, w + t1 - 1), cfg.noise_sigma)
    n2 = gaussian_noise(rng, (c, h + t2 - 1, w + t2 - 1), cfg.noise_sigma)
    return PairInputs(lat, k1, k2, n1, n2)
