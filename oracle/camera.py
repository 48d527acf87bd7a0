"""Camera side of the coprime blur scheme (Section 3, "Blur Kernel Selection"
and the cascaded pair), FP64 -- test infrastructure like the rest of the
package.

Per frame, a new pair of random square kernels is drawn; a pair is kept when
it passes the coprimality test (the reading of the paper's condition that the
two kernels, as bivariate polynomials, have a degree-0 GCD: at every sample
w^j of both evaluation orders the univariate kernel polynomials share no root,
sigma_min / sigma_max of their Sylvester matrix above a tolerance, and one of
them keeps full degree), else it is redrawn.  Random numbers come from
Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC 2011), written here from its published definition, so that a
device generator implementing the same definition draws the same kernels.
"""
from __future__ import annotations

import numpy as np

from .cbp_oracle import blur_full, root_powers, sylvester_system

_M0, _M1 = 0xD2511F53, 0xCD9E8D57          # Philox-4x32 multipliers
_W0, _W1 = 0x9E3779B9, 0xBB67AE85          # Weyl key increments
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Ten rounds of Philox-4x32 on a 4-word counter with a 2-word key."""
    c0, c1, c2, c3 = (int(x) & _MASK for x in ctr)
    k0, k1 = (int(x) & _MASK for x in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & _MASK, p1 & _MASK, ((p0 >> 32) ^ c3 ^ k1) & _MASK, \
            p0 & _MASK
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def draw_kernel(seed: int, frame: int, kind: int, attempt: int, t: int) -> np.ndarray:
    """Kernel `kind` (0, 1: the pair; 2, 3: the cascade's pair) of `frame` at
    redraw `attempt`: t x t entries uniform in (0, 1], normalised to unit sum.
    Entry e is word e mod 4 of Philox(counter = (e // 4, frame, kind * 256 +
    attempt, 0), key = seed); the uniform is (word + 1) 2^-32; the sum is
    taken in entry order."""
    key = (seed & _MASK, (seed >> 32) & _MASK)
    n = t * t
    u = np.empty(n, dtype=np.float64)
    for b in range((n + 3) // 4):
        words = philox4x32_10((b, frame, kind * 256 + attempt, 0), key)
        for i in range(4):
            e = 4 * b + i
            if e < n:
                u[e] = (float(words[i]) + 1.0) * 2.0 ** -32
    s = 0.0
    for v in u:
        s += v
    return (u / s).reshape(t, t)


def coprime_ratios(k1: np.ndarray, k2: np.ndarray, m: int):
    """sigma_min / sigma_max of the Sylvester matrix of the univariate kernel
    polynomials k1(., w^j), k2(., w^j) at every sample j < m of both evaluation
    orders (rows: evaluation along z2; columns: along z1), and whether one of
    the two keeps full degree there (leading coefficient above 1e-12 of its
    polynomial's norm).  The square Sylvester matrix is the cofactor system of
    the size scan at t1 - 1, t2 - 1: singular exactly when a root is shared."""
    t1, t2 = k1.shape[0], k2.shape[0]
    out = []
    for order in (0, 1):
        w1 = root_powers(t1, m)
        w2 = root_powers(t2, m)
        a_all = (k1 @ w1) if order == 0 else (k1.T @ w1)      # (t1, m): a_j[p]
        b_all = (k2 @ w2) if order == 0 else (k2.T @ w2)
        for j in range(m):
            a, b = a_all[:, j], b_all[:, j]
            full = abs(a[-1]) > 1e-12 * np.linalg.norm(a) or abs(b[-1]) > 1e-12 * np.linalg.norm(b)
            if t1 == 1 or t2 == 1:
                out.append((1.0, full))
                continue
            sv = np.linalg.svd(sylvester_system(a[None], b[None], t1 - 1, t2 - 1), compute_uv=False)
            out.append((sv[-1] / sv[0], full))
    return out


def is_coprime(k1, k2, m: int, tol: float = 1e-7) -> bool:
    return all(r > tol and full for r, full in coprime_ratios(k1, k2, m))


def draw_pair(seed: int, frame: int, t1: int, t2: int, m: int, kinds=(0, 1), max_attempts: int = 8,
              tol: float = 1e-7):
    """The first attempt whose pair passes the coprimality test; returns
    (k1, k2, attempt), or the last attempt's pair with attempt = -1."""
    for a in range(max_attempts):
        k1 = draw_kernel(seed, frame, kinds[0], a, t1)
        k2 = draw_kernel(seed, frame, kinds[1], a, t2)
        if is_coprime(k1, k2, m, tol):
            return k1, k2, a
    return k1, k2, -1


def encrypt(latent: np.ndarray, seed: int, frame: int, t1: int, t2: int, m: int | None = None,
            cascade: tuple[int, int] | None = None, max_attempts: int = 8, tol: float = 1e-7):
    """Encrypt one frame (Section 3): public stream B1 = L (x) K1, private
    stream B2 = L (x) K2 (Eq. 1, no noise here); with `cascade` = (t3, t4),
    the public stream is blurred again by a second coprime pair,
    C1 = B1 (x) K3, C2 = B1 (x) K4 (the cascaded pair).  latent (C, H, W)."""
    m = m or max(t1, t2)
    k1, k2, a = draw_pair(seed, frame, t1, t2, m, (0, 1), max_attempts, tol)
    out = {"k1": k1, "k2": k2, "attempt": a,
           "b1": np.stack([blur_full(ch, k1) for ch in latent]),
           "b2": np.stack([blur_full(ch, k2) for ch in latent])}
    if cascade:
        t3, t4 = cascade
        k3, k4, a2 = draw_pair(seed, frame, t3, t4, max(t3, t4), (2, 3), max_attempts, tol)
        out.update({"k3": k3, "k4": k4, "attempt_cascade": a2,
                    "c1": np.stack([blur_full(ch, k3) for ch in out["b1"]]),
                    "c2": np.stack([blur_full(ch, k4) for ch in out["b1"]])})
    return out
