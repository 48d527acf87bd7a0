"""Latent-frame, blur-kernel and noise generators (see the package docstring)."""
from __future__ import annotations

import math

import numpy as np

N_BLOBS = 20
BLOB_FLOOR = 0.05


def _rng(seed_or_rng) -> np.random.Generator:
    if isinstance(seed_or_rng, np.random.Generator):
        return seed_or_rng
    return np.random.Generator(np.random.PCG64(int(seed_or_rng)))


def blob_params(rng: np.random.Generator, h: int, w: int) -> np.ndarray:
    """Draw the 20 blobs of one channel: rows (amplitude, sigma, cx, cy)."""
    a = rng.uniform(0.0, 1.0, N_BLOBS)
    sigma = rng.uniform(2.0, 10.0, N_BLOBS)
    cx = rng.uniform(0.0, w, N_BLOBS)
    cy = rng.uniform(0.0, h, N_BLOBS)
    return np.stack([a, sigma, cx, cy], axis=1)


def blob_latent(seed_or_rng, h: int, w: int, channels: int = 1,
                dtype=np.float64) -> np.ndarray:
    """Latent frame(s) of shape (channels, h, w): 20 Gaussian blobs + U[0,0.05].

    Channels are drawn one after the other from the same generator (blob
    parameters, then the per-pixel floor).
    """
    rng = _rng(seed_or_rng)
    out = np.empty((channels, h, w), dtype=np.float64)
    for ch in range(channels):
        params = blob_params(rng, h, w)
        img = np.zeros((h, w), dtype=np.float64)
        for a, sigma, cx, cy in params:
            rad = int(math.ceil(8.0 * sigma))
            y0, y1 = max(0, int(math.floor(cy)) - rad), min(h, int(math.ceil(cy)) + rad + 1)
            x0, x1 = max(0, int(math.floor(cx)) - rad), min(w, int(math.ceil(cx)) + rad + 1)
            if y0 >= y1 or x0 >= x1:
                continue
            yy = np.arange(y0, y1, dtype=np.float64)[:, None] - cy
            xx = np.arange(x0, x1, dtype=np.float64)[None, :] - cx
            img[y0:y1, x0:x1] += a * np.exp(-(xx * xx + yy * yy) / (2.0 * sigma * sigma))
        img += rng.uniform(0.0, BLOB_FLOOR, (h, w))
        out[ch] = img
    return out.astype(dtype, copy=False)


def uniform_kernel(seed_or_rng, t: int) -> np.ndarray:
    """t x t kernel with U[0,1] entries, normalised to unit sum."""
    rng = _rng(seed_or_rng)
    k = rng.uniform(0.0, 1.0, (t, t))
    return k / k.sum()


def _gaussian_part(rng: np.random.Generator, t: int) -> np.ndarray:
    sx = rng.uniform(t / 6.0, t / 3.0)
    sy = rng.uniform(t / 6.0, t / 3.0)
    ang = rng.uniform(0.0, math.pi)
    c = (t - 1) / 2.0
    p = np.arange(t, dtype=np.float64)[:, None] - c      # row offset (y)
    q = np.arange(t, dtype=np.float64)[None, :] - c      # column offset (x)
    xr = math.cos(ang) * q + math.sin(ang) * p
    yr = -math.sin(ang) * q + math.cos(ang) * p
    g = np.exp(-0.5 * (xr * xr / (sx * sx) + yr * yr / (sy * sy)))
    return g / g.sum()


def _motion_part(rng: np.random.Generator, t: int) -> np.ndarray:
    c = (t - 1) / 2.0
    x, y = c, c
    heading = rng.uniform(0.0, 2.0 * math.pi)
    k = np.zeros((t, t), dtype=np.float64)

    def splat(px: float, py: float) -> None:
        x0, y0 = int(math.floor(px)), int(math.floor(py))
        fx, fy = px - x0, py - y0
        for dy, wy in ((0, 1.0 - fy), (1, fy)):
            for dx, wx in ((0, 1.0 - fx), (1, fx)):
                yy, xx = y0 + dy, x0 + dx
                if 0 <= yy < t and 0 <= xx < t:
                    k[yy, xx] += wy * wx

    splat(x, y)
    for _ in range(4 * t):
        heading += rng.normal(0.0, 0.5)
        x = min(max(x + math.cos(heading), 0.0), t - 1.0)
        y = min(max(y + math.sin(heading), 0.0), t - 1.0)
        splat(x, y)
    return k / k.sum()


def mixture_kernel(seed_or_rng, t: int) -> np.ndarray:
    """Gaussian + random-walk motion mixture kernel, normalised to unit sum."""
    rng = _rng(seed_or_rng)
    w = rng.uniform(0.3, 0.7)
    g = _gaussian_part(rng, t)
    mo = _motion_part(rng, t)
    k = w * g + (1.0 - w) * mo
    return k / k.sum()


def _sample_polys(k: np.ndarray, m: int, axis: int) -> np.ndarray:
    """Univariate coefficient vectors of k with the other variable at exp(-2 pi i j/m).

    axis=1 substitutes the column variable (rows stay as coefficients);
    axis=0 substitutes the row variable.  Returns (m, t).
    """
    t = k.shape[0]
    j = np.arange(m)[:, None]
    q = np.arange(t)[None, :]
    w = np.exp(-2j * np.pi * ((j * q) % m) / m)        # (m, t)
    if axis == 1:
        return w @ k.T        # [j][p] = sum_q k[p][q] w^{jq}
    return w @ k              # [i][q] = sum_p k[p][q] w^{ip}


def pair_is_coprime(k1: np.ndarray, k2: np.ndarray, m: int,
                    min_sep: float = 1e-3, min_lead: float = 1e-9) -> bool:
    """Generator acceptance test (no common root at any sample, full degree).

    For each evaluation order and each of the m samples, the two univariate
    polynomials must (a) not both lose their leading coefficient and (b) have
    root sets separated by at least ``min_sep`` (relative to 1 + |root|).
    """
    for axis in (0, 1):
        p1s = _sample_polys(k1, m, axis)
        p2s = _sample_polys(k2, m, axis)
        for p1, p2 in zip(p1s, p2s):
            scale = max(np.abs(p1).max(), np.abs(p2).max())
            if scale == 0.0:
                return False
            if max(abs(p1[-1]), abs(p2[-1])) < min_lead * scale:
                return False
            # numpy.roots wants the highest power first
            r1 = np.roots(p1[::-1]) if len(p1) > 1 else np.zeros(0)
            r2 = np.roots(p2[::-1]) if len(p2) > 1 else np.zeros(0)
            if r1.size and r2.size:
                d = np.abs(r1[:, None] - r2[None, :])
                rel = d / (1.0 + np.minimum(np.abs(r1)[:, None], np.abs(r2)[None, :]))
                if rel.min() < min_sep:
                    return False
    return True


def draw_kernel_pair(seed_or_rng, t1: int, t2: int, m: int, family: str = "uniform",
                     max_tries: int = 100):
    """Draw (K1, K2) of the given family, redrawn until ``pair_is_coprime``."""
    rng = _rng(seed_or_rng)
    make = {"uniform": uniform_kernel, "mixture": mixture_kernel}[family]
    for _ in range(max_tries):
        k1 = make(rng, t1)
        k2 = make(rng, t2)
        if pair_is_coprime(k1, k2, m):
            return k1, k2
    raise RuntimeError("no coprime kernel pair found")


def gaussian_noise(seed_or_rng, shape, sigma: float) -> np.ndarray:
    """N(0, sigma^2) noise of the given shape (zeros when sigma == 0)."""
    if sigma == 0.0:
        return np.zeros(shape, dtype=np.float64)
    rng = _rng(seed_or_rng)
    return rng.normal(0.0, sigma, shape)
