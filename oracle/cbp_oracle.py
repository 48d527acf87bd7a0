"""Plain FP64 restatement of the CBP method (test infrastructure, see package doc).

Notation (follows the paper's Eq. 1-4 and Sections 4-5):
  B_k[r][c]   blurred frame k (k = 1, 2); r indexes rows (the z1 direction),
              c indexes columns (the z2 direction), Eq. 3.
  K_k         t_k x t_k blur kernel; latent L is H x W; B_k = L (x) K_k is the
              full convolution, (H + t_k - 1) x (W + t_k - 1), Eq. 1.
  omega       exp(-2 pi i / M); samples are omega^j, j = 0..M-1, on the unit
              circle (Section 5: the evaluation is an M-point DFT).
Arrays carry a leading channel axis; the kernels are shared by all channels
and the per-sample systems stack the channels' rows.

Readings where the paper is silent (the citing design notes list them all):
  * M = max(t1, t2) samples by default; samples use the forward-DFT sign.
  * The per-sample 1D GCD cofactors are the null vector of the Sylvester
    (convolution) matrix of the identity b1 * k2 - b2 * k1 = 0 (Eq. 4), taken
    as the right singular vector of the smallest singular value and scaled to
    unit 2-norm.
  * Scale fix (Section 4, last paragraph; Section 5): unknown per-sample
    factors gamma_j (z2-first order) and delta_i (z1-first order) solve
    gamma_j * A_k[i][j] - delta_i * B_k[i][j] = 0 for both kernels in the least
    squares sense (null vector by SVD); the two estimates are averaged and each
    kernel spectrum is normalised so that its [0][0] entry (the kernel sum) is 1.
  * Latent recovery uses the dual-kernel Fourier formula
    (conj(K1)B1 + conj(K2)B2) / (|K1|^2 + |K2|^2 + eps) on the smallest
    7-smooth grid that holds the larger blurred frame, cropped at (0, 0).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- sampling ---
def root_powers(n: int, m: int, sign: int = -1) -> np.ndarray:
    """w[c][j] = exp(sign * 2 pi i * (c*j mod m) / m), shape (n, m).

    The unit-circle samples of Section 5 ("points around the unit circle");
    the exponent is reduced mod m before the exponential for accuracy.
    """
    c = np.arange(n, dtype=np.int64)[:, None]
    j = np.arange(m, dtype=np.int64)[None, :]
    return np.exp(sign * 2j * np.pi * ((c * j) % m) / m)


# ------------------------------------------------------------ forward model ---
def blur_full(latent: np.ndarray, kernel: np.ndarray) -> np.ndarray:
    """Eq. 1 without noise: B[r][c] = sum_{p,q} L[r-p][c-q] K[p][q], full size."""
    h, w = latent.shape
    t = kernel.shape[0]
    out = np.zeros((h + t - 1, w + t - 1), dtype=np.float64)
    for p in range(t):
        for q in range(t):
            out[p:p + h, q:q + w] += kernel[p, q] * latent
    return out


def blur_pair(latent: np.ndarray, k1: np.ndarray, k2: np.ndarray,
              noise1: np.ndarray | None = None, noise2: np.ndarray | None = None):
    """The coprime blurred pair of Section 3: B_k = L (x) K_k + N_k per channel."""
    b1 = np.stack([blur_full(ch, k1) for ch in latent])
    b2 = np.stack([blur_full(ch, k2) for ch in latent])
    if noise1 is not None:
        b1 = b1 + noise1
    if noise2 is not None:
        b2 = b2 + noise2
    return b1, b2


# ------------------------------------------------------- polynomial evaluation
def evaluate_z2(b: np.ndarray, m: int) -> np.ndarray:
    """Eq. 3 with z2 = omega^j: P[ch][j][r] = sum_c B[ch][r][c] omega^(j c).

    Row j holds the z1-coefficients of b(z1, omega^j) (Section 4: evaluation
    along one direction turns the 2D problem into 1D ones).  Shape (C, m, H_B).
    """
    w = root_powers(b.shape[2], m)                  # (W_B, m)
    return np.stack([(ch @ w).T for ch in b])


def evaluate_z1(b: np.ndarray, m: int) -> np.ndarray:
    """Eq. 3 with z1 = omega^i: P[ch][i][c] = sum_r B[ch][r][c] omega^(i r).

    Row i holds the z2-coefficients of b(omega^i, z2).  Shape (C, m, W_B).
    """
    w = root_powers(b.shape[1], m)                  # (H_B, m)
    return np.stack([w.T @ ch for ch in b])


# ------------------------------------------------------ per-sample 1D problem
def convolution_matrix(b: np.ndarray, t: int) -> np.ndarray:
    """C_t(b)[r][p] = b[r - p]: (len(b) + t - 1) x t, so C_t(b) u = b * u."""
    n = b.shape[0]
    out = np.zeros((n + t - 1, t), dtype=np.complex128)
    for p in range(t):
        out[p:p + n, p] = b
    return out


def sylvester_system(b1s, b2s, t1: int, t2: int) -> np.ndarray:
    """S = [-C_t1(b2) | C_t2(b1)] stacked over channels.

    S [u; v] = b1 * v - b2 * u, which vanishes for u = k1, v = k2 because
    b1 k2 = l k1 k2 = b2 k1 (Eq. 4: k1, k2 are the cofactors of the GCD l).
    """
    blocks = [np.hstack([-convolution_matrix(b2, t1), convolution_matrix(b1, t2)])
              for b1, b2 in zip(b1s, b2s)]
    return np.vstack(blocks)


def null_vector(s: np.ndarray):
    """Right singular vector of the smallest singular value (unit 2-norm).

    Returns (x, singular values in descending order).  Section 5 factors the
    per-sample matrices by SVD.
    """
    _, sv, vh = np.linalg.svd(s, full_matrices=False)
    return vh[-1].conj(), sv


def cofactors_pass(p1: np.ndarray, p2: np.ndarray, t1: int, t2: int):
    """One evaluation order: the 1D cofactor pair at every sample (Section 4).

    p1, p2: (C, M, len) sample polynomials of B1 and B2.  Returns
    X (M, t1 + t2) -- X[s] = [u; v] with u ~ k1 and v ~ k2 at sample s -- and
    the singular values (M, t1 + t2) of every sample's system.
    """
    m = p1.shape[1]
    n = t1 + t2
    xs = np.zeros((m, n), dtype=np.complex128)
    svs = np.zeros((m, n), dtype=np.float64)
    for s in range(m):
        sys_s = sylvester_system(p1[:, s, :], p2[:, s, :], t1, t2)
        xs[s], svs[s] = null_vector(sys_s)
    return xs, svs


# ------------------------------------------------------- 2D kernel estimation
def lift(x_z2: np.ndarray, x_z1: np.ndarray, t1: int, t2: int, m: int):
    """Evaluate the 1D cofactors on the unit circle (Section 5, 2D kernel estimation).

    z2-first order: A_k[i][j] = sum_p u_{k,j}[p] omega^(i p)  (= c_j K_k^[i][j])
    z1-first order: B_k[i][j] = sum_q u_{k,i}[q] omega^(j q)  (= d_i K_k^[i][j])
    where u_{1,s} = X[s][:t1], u_{2,s} = X[s][t1:].  Returns (A, B), each (2, M, M).
    """
    a = np.zeros((2, m, m), dtype=np.complex128)
    b = np.zeros((2, m, m), dtype=np.complex128)
    for k, (lo, t) in enumerate(((0, t1), (t1, t2))):
        w = root_powers(t, m)                        # (t, M): w[p][i] = omega^(ip)
        a[k] = (x_z2[:, lo:lo + t] @ w).T            # [i][j]
        b[k] = x_z1[:, lo:lo + t] @ w                # [i][j]
    return a, b


def scale_least_squares(a: np.ndarray, b: np.ndarray):
    """Least-squares scale fix between the two evaluation orders (Sections 4-5).

    Unknowns (gamma_0..gamma_{M-1}, delta_0..delta_{M-1}); one equation per
    kernel k and entry (i, j): gamma_j A_k[i][j] - delta_i B_k[i][j] = 0.
    The solution is the null vector (smallest right singular vector) of this
    2M^2 x 2M system.  Returns (gamma, delta, singular values).
    """
    m = a.shape[1]
    rows = []
    for k in range(a.shape[0]):                      # the kernels whose equations enter
        for i in range(m):
            for j in range(m):
                row = np.zeros(2 * m, dtype=np.complex128)
                row[j] = a[k, i, j]
                row[m + i] = -b[k, i, j]
                rows.append(row)
    theta, sv = null_vector(np.array(rows))
    return theta[:m], theta[m:], sv


def scale_least_squares_k1(a: np.ndarray, b: np.ndarray):
    """The paper's k1-only pipeline (Section 4 recovers the cofactor k1 and
    divides B1 by K1): the scale fix of `scale_least_squares` with kernel 1's
    equations only, gamma_j A_1[i][j] - delta_i B_1[i][j] = 0 (M^2 equations).
    Returns (gamma, delta, singular values)."""
    return scale_least_squares(a[:1], b[:1])


def scale_support(a: np.ndarray, t1: int, t2: int):
    """Single-pass scale fix from the kernels' support (a reading of Section
    5's remark that the M x M estimates hold kernels of size t < M): with the
    z2-first lift A_k[i][j] = c_j K_k^[i][j] only, the inverse DFT along j of
    gamma_j A_k[i][j] must vanish at the columns q >= t_k the kernel does not
    occupy:  sum_j gamma_j A_k[i][j] omega^(-j q) = 0  for k = 1, 2, every i and
    t_k <= q < M.  gamma is the null vector of this 2 M (M - t) x M system (by
    SVD); needs M > max(t1, t2).  Returns (gamma, singular values)."""
    m = a.shape[1]
    if m <= max(t1, t2):
        raise ValueError("the support constraint needs M > max(t1, t2)")
    v = root_powers(m, m, sign=+1)                   # v[j][q] = omega^(-jq)
    rows = []
    for k, t in ((0, t1), (1, t2)):
        for i in range(m):
            for q in range(t, m):
                rows.append(a[k, i, :] * v[:, q])
    gamma, sv = null_vector(np.array(rows))
    return gamma, sv


def kernel_spectra_support(a: np.ndarray, gamma: np.ndarray):
    """X_k[i][j] = gamma_j A_k[i][j], normalised so that X_k[0][0] = 1."""
    x = gamma[None, None, :] * a
    return x / x[:, :1, :1]


def kernel_spectra(a: np.ndarray, b: np.ndarray, gamma: np.ndarray, delta: np.ndarray):
    """Average the two rescaled estimates and normalise each to unit sum (Section 5).

    X_k[i][j] = (gamma_j A_k[i][j] + delta_i B_k[i][j]) / 2, then X_k /= X_k[0][0].
    """
    x = 0.5 * (gamma[None, None, :] * a + delta[None, :, None] * b)
    return x / x[:, :1, :1]


def kernels_from_spectra(xk: np.ndarray, t: int):
    """Inverse M x M DFT of a kernel spectrum (Section 5, "inverse FFT").

    K_full[p][q] = (1/M^2) sum_{i,j} X[i][j] omega^(-(i p + j q)), p, q < M.
    Returns (real part of the leading t x t block, complex K_full).
    """
    m = xk.shape[0]
    v = root_powers(m, m, sign=+1)                   # v[i][p] = omega^(-ip)
    full = (v.T @ xk @ v) / (m * m)
    return full[:t, :t].real.copy(), full


# ------------------------------------------------------------- deconvolution
def fft_grid_size(n: int) -> int:
    """Smallest integer >= n whose prime factors are all in {2, 3, 5, 7}."""
    k = max(int(n), 1)
    while True:
        r = k
        for p in (2, 3, 5, 7):
            while r % p == 0:
                r //= p
        if r == 1:
            return k
        k += 1


def deconvolve_dual(b1: np.ndarray, b2: np.ndarray, k1: np.ndarray, k2: np.ndarray,
                    h: int, w: int, eps: float, ph: int | None = None, pw: int | None = None):
    """Dual-kernel Fourier deconvolution (Section 4 divides by K1 in the Fourier domain;
    this uses both kernels): I^ = (conj(K1^) B1^ + conj(K2^) B2^) / (|K1^|^2 + |K2^|^2 + eps).

    All spectra are 2D DFTs of the zero-padded arrays on a ph x pw grid (default:
    smallest 7-smooth sizes holding the larger blurred frame).  The latent is the
    real part of the inverse DFT, cropped to [0:h, 0:w].  Returns (C, h, w).
    """
    if ph is None:
        ph = fft_grid_size(max(b1.shape[1], b2.shape[1]))
    if pw is None:
        pw = fft_grid_size(max(b1.shape[2], b2.shape[2]))
    fk1 = np.fft.fft2(k1, s=(ph, pw))
    fk2 = np.fft.fft2(k2, s=(ph, pw))
    den = np.abs(fk1) ** 2 + np.abs(fk2) ** 2 + eps
    if eps == 0.0 and den.min() < 1e-280:
        raise ZeroDivisionError("dual-kernel denominator vanishes with eps = 0")
    out = np.zeros((b1.shape[0], h, w), dtype=np.float64)
    for ch in range(b1.shape[0]):
        fb1 = np.fft.fft2(b1[ch], s=(ph, pw))
        fb2 = np.fft.fft2(b2[ch], s=(ph, pw))
        lat = np.fft.ifft2((np.conj(fk1) * fb1 + np.conj(fk2) * fb2) / den)
        out[ch] = lat[:h, :w].real
    return out


# --------------------------------------------------------------- pipelines ---
def estimate_kernels(b1: np.ndarray, b2: np.ndarray, t1: int, t2: int, m: int | None = None,
                     scale: str = "ls"):
    """Blind recovery of (K1, K2) from a coprime blurred pair, in the paper's order.

    b1, b2: (C, H_B1, W_B1) and (C, H_B2, W_B2).  Returns a dict of every
    intermediate (sample polynomials, per-sample cofactors and singular values,
    lifted spectra, scale factors, kernel spectra, kernels, diagnostics).
    """
    b1 = np.asarray(b1, dtype=np.float64)
    b2 = np.asarray(b2, dtype=np.float64)
    if b1.ndim == 2:
        b1, b2 = b1[None], b2[None]
    if m is None:
        m = max(t1, t2)
    out = {"m": m}
    # Evaluation along z2 first, then along z1 (Section 4, both orders).
    out["p_z2_1"], out["p_z2_2"] = evaluate_z2(b1, m), evaluate_z2(b2, m)
    out["p_z1_1"], out["p_z1_2"] = evaluate_z1(b1, m), evaluate_z1(b2, m)
    out["x_z2"], out["sv_z2"] = cofactors_pass(out["p_z2_1"], out["p_z2_2"], t1, t2)
    out["x_z1"], out["sv_z1"] = cofactors_pass(out["p_z1_1"], out["p_z1_2"], t1, t2)
    out["a_hat"], out["b_hat"] = lift(out["x_z2"], out["x_z1"], t1, t2, m)
    if scale == "support":
        # single pass: the z2-first lift and the support constraint only
        out["gamma"], out["sv_scale"] = scale_support(out["a_hat"], t1, t2)
        out["x_k"] = kernel_spectra_support(out["a_hat"], out["gamma"])
    elif scale == "k1":
        out["gamma"], out["delta"], out["sv_scale"] = scale_least_squares_k1(out["a_hat"], out["b_hat"])
        x1 = kernel_spectra(out["a_hat"][:1], out["b_hat"][:1], out["gamma"], out["delta"])
        out["x_k"] = np.concatenate([x1, np.full_like(x1, np.nan)])
    else:
        out["gamma"], out["delta"], out["sv_scale"] = scale_least_squares(out["a_hat"], out["b_hat"])
        out["x_k"] = kernel_spectra(out["a_hat"], out["b_hat"], out["gamma"], out["delta"])
    out["k1"], out["k1_full"] = kernels_from_spectra(out["x_k"][0], t1)
    if scale == "k1":
        out["k2"] = out["k2_full"] = None
    else:
        out["k2"], out["k2_full"] = kernels_from_spectra(out["x_k"][1], t2)
    sv = np.concatenate([out["sv_z2"], out["sv_z1"]])
    gap = sv[:, -2] / sv[:, 0]
    out["diag"] = {
        "sigma_gap": gap,                            # sigma_{n-1} / sigma_1 per sample
        "sigma_min": sv[:, -1] / sv[:, 0],           # sigma_n / sigma_1 per sample
        "kappa": float(np.max(1.0 / gap)),
        "gap_min": float(gap.min()),
        "flagged_samples": int(np.sum(gap < 1e-8)),
        "scale_resid": float(out["sv_scale"][-1] / out["sv_scale"][0]),
    }
    return out


def deblur_pair(b1, b2, t1: int, t2: int, m: int | None = None, eps: float = 1e-4,
                k1=None, k2=None, ph: int | None = None, pw: int | None = None, scale: str = "ls"):
    """Kernels (estimated unless given) and the latent frame of one pair (Sections 4-5).
    scale: "ls" (both kernels' two-order least squares, dual-kernel division),
    "support" (single-pass support-constrained scale fix), "k1" (the paper's
    k1-only pipeline: kernel 1's scale fix, B1 divided by K1)."""
    b1 = np.asarray(b1, dtype=np.float64)
    b2 = np.asarray(b2, dtype=np.float64)
    if b1.ndim == 2:
        b1, b2 = b1[None], b2[None]
    out = {}
    if k1 is None or (k2 is None and scale != "k1"):
        out = estimate_kernels(b1, b2, t1, t2, m, scale)
        k1, k2 = out["k1"], out["k2"]
    h = b1.shape[1] - t1 + 1
    w = b1.shape[2] - t1 + 1
    if scale == "k1":
        k2 = np.zeros((t2, t2))                      # single-kernel form: B1 / K1
    out["latent"] = deconvolve_dual(b1, b2, k1, k2, h, w, eps, ph, pw)
    return out


# ------------------------------------------------------- kernel-size estimation
def plane_sums(b: np.ndarray):
    """The z = 1 samples of both evaluation orders (Eq. 3 at z2 = 1 and z1 = 1):
    row sums (C, H_B) and column sums (C, W_B) of a frame."""
    b = np.asarray(b, dtype=np.float64)
    return b.sum(axis=2), b.sum(axis=1)


def size_ratios(b1: np.ndarray, b2: np.ndarray, t_min: int, t_max: int):
    """Singularity test of the kernel-degree step (Section 4: the degree is read
    from the singularity of the cofactor system; Section 5: square candidates in
    a fixed range).  Under full convolution the blurred sizes fix d = t1 - t2;
    for each candidate t1' in [t_min, t_max] (t2' = t1' - d) the Sylvester
    system of the z = 1 samples is built for both evaluation orders and its
    sigma_min / sigma_max taken by SVD.  The system has a null vector exactly
    when t1' >= t1 (then u = k1 s, v = k2 s for any s of degree t1' - t1), so
    the ratio drops to the noise floor at the true size.  Returns
    (d, {t1': max over the two orders of sigma_min / sigma_max})."""
    b1 = np.asarray(b1, dtype=np.float64)
    b2 = np.asarray(b2, dtype=np.float64)
    if b1.ndim == 2:
        b1, b2 = b1[None], b2[None]
    d = b1.shape[1] - b2.shape[1]
    if b1.shape[2] - b2.shape[2] != d:
        raise ValueError("blurred sizes disagree on t1 - t2")
    r1, c1 = plane_sums(b1)
    r2, c2 = plane_sums(b2)
    out = {}
    for t1 in range(t_min, t_max + 1):
        t2 = t1 - d
        if t2 < 1 or t1 < 1:
            continue
        worst = 0.0
        for p1, p2 in ((r1, r2), (c1, c2)):
            sv = np.linalg.svd(sylvester_system(p1, p2, t1, t2), compute_uv=False)
            worst = max(worst, sv[-1] / sv[0])
        out[t1] = worst
    return d, out


def estimate_size(b1, b2, t_min: int = 1, t_max: int = 32, tol: float = 1e-6):
    """Kernel degree (Section 4, Section 5): the smallest candidate whose system
    is numerically singular (sigma_min / sigma_max <= tol); when none is, the
    largest candidate (Section 5 falls back to its largest size).  Returns
    (t1, t2, found, ratios)."""
    d, ratios = size_ratios(b1, b2, t_min, t_max)
    if not ratios:
        raise ValueError("no valid candidate size")
    for t1 in sorted(ratios):
        if ratios[t1] <= tol:
            return t1, t1 - d, True, ratios
    t1 = max(ratios)
    return t1, t1 - d, False, ratios


# ------------------------------------------------------ multi-level security
def truncate_lsb(b: np.ndarray, bits: int, drop: int) -> np.ndarray:
    """Multi-level access to the private stream (Section 3, "Multi-level
    Security"): a lower clearance level receives the blurred frames with the
    least significant bits removed.  Reading: intensities in [0, 1] are coded
    as unsigned integers of `bits` bits, code = rint(x (2^bits - 1)) clamped to
    [0, 2^bits - 1]; level `drop` clears the code's `drop` lowest bits; the
    value it sees is code / (2^bits - 1).  Computed in double precision."""
    if not (1 <= bits <= 30 and 0 <= drop < bits):
        raise ValueError("need 1 <= bits <= 30 and 0 <= drop < bits")
    top = float((1 << bits) - 1)
    code = np.clip(np.rint(np.asarray(b, dtype=np.float64) * top), 0.0, top).astype(np.int64)
    code &= ~np.int64((1 << drop) - 1)
    return code.astype(np.float64) / top
