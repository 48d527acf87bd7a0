/*
 * cbp.h -- C ABI of libcbp, a single-GPU (sm_103a) implementation of Coprime
 * Blurred Pair (CBP) deblurring: Thorpe, Li, Li, Yu, Saunders, Yu, "A Co-Prime
 * Blur Scheme for Data Security in Video Surveillance" (arXiv 1203.4874).
 *
 * Problem (Section 4, Eq. 1 and Eq. 4): two frames of one scene, B1 = L (x) K1
 * and B2 = L (x) K2 (full 2D convolution plus sensor noise), blurred by two
 * unknown kernels that are coprime as bivariate polynomials (Section 3).
 * Recover K1, K2 blindly and then the latent frame L.
 *
 * Conventions for every entry point:
 *   - All calls are asynchronous on the given CUDA stream (`stream` is a
 *     cudaStream_t passed as void*; NULL is the legacy default stream) unless
 *     stated otherwise.  Host-side validation happens before anything is
 *     enqueued; a negative return value means nothing was enqueued.
 *   - Frame, kernel and latent buffers are owned by the caller.  Device
 *     pointers must stay valid until the stream reaches the call's work.
 *   - A context owns its device workspace, which is counted against the HBM
 *     budget given to cbp_create().  Calls on one context that use its
 *     workspace (estimate / deblur / forward) must be ordered on one stream, or
 *     the caller must synchronise between them.
 *   - No C++ exception crosses the ABI.  Negative cbp_status values are
 *     errors, positive values are warnings, 0 is success.
 *   - Arrays are row-major.  A frame batch is addressed as
 *       data[f * frame_stride + ch * chan_stride + r * row_stride + col]
 *     in elements of its dtype.
 */
#ifndef CBP_H_
#define CBP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cbp_status {
  CBP_OK = 0,
  CBP_WARN_ILL_CONDITIONED = 1, /* some sample had sigma_{n-1}/sigma_1 < 1e-8  */
  CBP_ERR_INVALID_ARG = -1,     /* bad pointer, size, dtype, NaN/Inf input     */
  CBP_ERR_SIZE_MISMATCH = -2,   /* blurred sizes inconsistent with t1, t2      */
  CBP_ERR_NOT_COPRIME = -3,     /* some sample had sigma_{n-1}/sigma_1 < 1e-13 */
  CBP_ERR_OOM = -4,             /* device allocation failed                    */
  CBP_ERR_CUDA = -5,            /* a CUDA runtime call failed                  */
  CBP_ERR_BUSY = -6,            /* stream request not finished yet             */
  CBP_ERR_TIMEOUT = -7,         /* wait limit reached                          */
  CBP_ERR_BUDGET = -8,          /* request exceeds the context's HBM budget    */
  CBP_ERR_UNSUPPORTED = -9      /* size beyond a documented library limit      */
} cbp_status;

typedef enum cbp_dtype { CBP_F32 = 0, CBP_F64 = 1 } cbp_dtype;

/* Arithmetic of the kernel-estimation path.
 *   FP64:  evaluation, Gram and per-sample solves in double precision (the
 *          per-sample eigen-solve runs in single precision and is refined to
 *          double precision against the double-precision Gram and two
 *          exact-residual steps).  Deconvolution in the frames' dtype.
 *   MIXED: evaluation with single-precision arithmetic (float frames are
 *          folded with an exact hi + lo float accumulation, samples kept in
 *          double); Gram of the samples other than z = 1 in single precision;
 *          eigen-solves in single precision refined in double precision (one
 *          exact-residual step); scale fix in double precision;
 *          deconvolution in single precision.
 *   LEARNED: a network proposal checked by the consistency residual, falling
 *          back to MIXED (see cbp_learned_*). */
typedef enum cbp_path { CBP_PATH_FP64 = 0, CBP_PATH_MIXED = 1, CBP_PATH_LEARNED = 2 } cbp_path;

/* A batch of n frames of one shape (one frame of each pair per batch entry). */
typedef struct cbp_frames {
  const void* data;     /* device pointer (host pointer with CBP_FLAG_HOST_IO) */
  int32_t n;            /* frames in the batch, >= 1                          */
  int32_t c;            /* channels, >= 1 (kernels are shared by channels)    */
  int32_t h, w;         /* rows, columns of each channel                      */
  cbp_dtype dtype;
  int64_t row_stride;   /* elements; 0 => w                                   */
  int64_t chan_stride;  /* elements; 0 => h * row_stride                      */
  int64_t frame_stride; /* elements; 0 => c * chan_stride                     */
} cbp_frames;

/* Flags of cbp_params.flags. */
#define CBP_FLAG_HOST_IO 1u      /* frames, kernels and latent are host buffers; the
                                    library stages them through device memory on the
                                    stream (pinned host memory keeps this async)    */
#define CBP_FLAG_KERNELS_IN 2u   /* k1, k2 are inputs: skip estimation, deconvolve */
#define CBP_FLAG_SINGLE_KERNEL 4u/* deconvolve B1 by K1 alone (Section 4) instead of
                                    the dual-kernel formula                         */
#define CBP_FLAG_KERNELS_F64 8u  /* k1, k2 buffers hold doubles whatever the frames'
                                    dtype (the FP64 path's full accuracy)           */
#define CBP_FLAG_K1_ONLY    16u  /* the paper's k1-only pipeline (Section 4: the
                                    cofactor k1, then B1 divided by K1): the scale
                                    fix from kernel 1's equations only, the
                                    single-kernel deconvolution; k2 is not written  */
#define CBP_FLAG_SCALE_SUPPORT 32u /* single-pass scale fix from the kernels'
                                    support: with m > max(t1, t2) the z2-first
                                    estimates' inverse DFT must vanish at columns
                                    q >= t_k; gamma_j is the null vector of those
                                    equations (the z1-first pass is not used).
                                    Needs m > max(t1, t2); excludes K1_ONLY        */
#define CBP_FLAG_OVERLAP_CALLS 64u /* with CBP_FLAG_HOST_IO: the call's input copies
                                    and kernels do not wait for earlier work on the
                                    stream, only for this context's previous call
                                    to be done with each chunk's buffers, so
                                    consecutive calls overlap (one's input copies
                                    beside another's tail).  The caller guarantees
                                    that nothing on the stream still writes the
                                    host input buffers.  Takes effect when the
                                    previous call on the context had the same
                                    chunk layout; results are unchanged          */

typedef struct cbp_params {
  int32_t t1, t2;     /* kernel sizes (square kernels), 1 <= t_k, t1 + t2 <= 64  */
  int32_t m;          /* unit-circle samples per direction; 0 => max(t1, t2);
                         must satisfy max(t1, t2) <= m <= 32                      */
  cbp_path path;
  double eps;         /* Wiener regulariser of the deconvolution, >= 0           */
  int32_t pad_h, pad_w; /* FFT grid; 0 => smallest 7-smooth >= larger blurred size */
  double accept_rho;  /* learned path: accept the proposal when rho <= accept_rho  */
  uint32_t flags;     /* CBP_FLAG_*                                              */
  int32_t reserved;
} cbp_params;

/* Candidate range and tolerance of the kernel-size scan (cbp_estimate_size). */
typedef struct cbp_size_params {
  int32_t t_min;      /* smallest candidate t1; 0 => 1                            */
  int32_t t_max;      /* largest candidate t1; 0 => 32 (capped by t1 + t2 <= 64 and
                         the frame size)                                           */
  double tol;         /* a candidate is singular when sigma_min / sigma_max <= tol;
                         0 => 1e-6                                                 */
} cbp_size_params;

/* Per-pair diagnostics, computed on the device (one entry per batch entry). */
typedef struct cbp_diag {
  double kappa_max;     /* max over samples of sigma_1 / sigma_{n-1}               */
  double gap_min;       /* min over samples of sigma_{n-1} / sigma_1               */
  double sigma_min_max; /* max over samples of sigma_n / sigma_1 (noise level)     */
  double scale_resid;   /* sigma_min / sigma_max of the scale least-squares system */
  double imag_ratio;    /* ||Im|| / ||Re|| of the inverse DFT of the kernel spectra */
  double support_ratio; /* energy of the inverse DFT outside t_k x t_k / total     */
  double rho;           /* learned path: ||B1*K2 - B2*K1|| / ||B1||                */
  int32_t flagged_samples; /* samples with sigma_{n-1}/sigma_1 < 1e-8              */
  int32_t used_fallback;   /* learned path: 1 if the GCD solve ran                 */
  int32_t pad_h, pad_w;    /* FFT grid used                                        */
  int32_t status;          /* cbp_status derived from the fields above             */
  int32_t hard_samples;    /* samples whose two smallest normal-matrix eigenvalues
                              are within 1e-4 of the largest (near-degenerate)  */
  double gpu_start_ms;     /* serving: the request's batch began / ended on the   */
  double gpu_end_ms;       /* device, ms after the engine started (CUDA events);
                              0 for the synchronous calls                          */
} cbp_diag;

typedef struct cbp_ctx cbp_ctx;

/* Create a context on `device` (made current for the call).  Device memory
 * the context allocates (workspaces, serving slots) never exceeds
 * hbm_budget_bytes (0 => 90% of the free memory at creation).
 * Errors: CBP_ERR_INVALID_ARG (out == NULL), CBP_ERR_CUDA (bad device). */
cbp_status cbp_create(cbp_ctx** out, int device, size_t hbm_budget_bytes);

/* Destroy a context: waits for its serving work, frees everything it owns. */
cbp_status cbp_destroy(cbp_ctx* ctx);

/* Human-readable name of a status code (static string, never NULL). */
const char* cbp_status_string(cbp_status s);

/* Device workspace one cbp_deblur_pair / cbp_estimate_kernels call with these
 * arguments needs (bytes, written to *bytes).  No device work. */
cbp_status cbp_workspace_size(const cbp_frames* b1, const cbp_frames* b2,
                              const cbp_params* params, size_t* bytes);

/* Kernel-size estimation for a batch of frame pairs (Section 4: the degree
 * of the blur kernels comes first, from the singularity of the cofactor
 * system; Section 5: a scan over square candidate sizes that falls back to
 * the largest when no candidate is singular).  Under full convolution the
 * blurred sizes fix d = t1 - t2 = H_B1 - H_B2 = W_B1 - W_B2 (else
 * CBP_ERR_SIZE_MISMATCH).  For every candidate t1' (t2' = t1' - d) the
 * Sylvester system of the z = 1 samples (row sums for the z2-first order,
 * column sums for the z1-first order; channels' rows stacked) is formed and
 * ratio(t1') = sigma_min / sigma_max taken, the larger of the two orders'; the
 * system has a null vector exactly when t1' >= t1.  The estimate is the
 * smallest candidate with ratio <= tol, else the largest candidate.
 * params: NULL or the candidate range and tolerance.
 * t1_out, t2_out: host arrays of n entries; found: NULL or host array of n
 * (1: a singular candidate was found, 0: the fallback); ratios: NULL or host
 * array [n][ncand] with ncand = t_max - t_min + 1 after the caps (-1 marks a
 * candidate the caps exclude) -- all filled by asynchronous copies on the
 * stream, valid after it is synchronised (pinned memory recommended).
 * *ncand_out: NULL or the number of candidates (set before returning).
 * Errors: CBP_ERR_INVALID_ARG, CBP_ERR_SIZE_MISMATCH, CBP_ERR_BUDGET,
 * CBP_ERR_OOM, CBP_ERR_CUDA. */
cbp_status cbp_estimate_size(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                             const cbp_size_params* params, int32_t* t1_out, int32_t* t2_out,
                             int32_t* found, double* ratios, int32_t* ncand_out, void* stream);

/* Blind kernel estimation for a batch of frame pairs (Sections 4-5):
 *   1. evaluation of both frames' z-polynomials at the m-th roots of unity in
 *      z2 (rows kept) and in z1 (columns kept) -- Eq. 3, Section 5's DFT;
 *   2. at every sample, the univariate cofactor pair (u, v) ~ (k1, k2) as the
 *      null vector of the Sylvester system b1*v - b2*u = 0 (Eq. 4), channels'
 *      rows stacked;
 *   3. lifting of the cofactors to two m x m estimates of the kernels' 2D DFT,
 *      least-squares fix of their per-sample scales, average, normalisation to
 *      unit kernel sum (Section 5);
 *   4. inverse m x m DFT to the spatial kernels.
 * b1: n frames of (H + t1 - 1) x (W + t1 - 1); b2: n frames of
 * (H + t2 - 1) x (W + t2 - 1); same n, c and dtype.
 * k1: device, n * t1 * t1 elements of b1's dtype (double with
 * CBP_FLAG_KERNELS_F64); k2: n * t2 * t2 (row-major).
 * diag: NULL or host array of n entries, filled by an asynchronous copy on the
 * stream (valid after the stream is synchronised; pinned memory recommended).
 * Errors: CBP_ERR_INVALID_ARG, CBP_ERR_SIZE_MISMATCH, CBP_ERR_UNSUPPORTED,
 * CBP_ERR_BUDGET, CBP_ERR_OOM, CBP_ERR_CUDA.  Device-detected conditions
 * (ill-conditioned or non-coprime samples, NaN/Inf input) are reported in
 * diag[i].status. */
cbp_status cbp_estimate_kernels(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                                const cbp_params* params, void* k1, void* k2,
                                cbp_diag* diag, void* stream);

/* Intermediates of the estimation path, for stage-by-stage checking.  Every
 * member is NULL (skipped) or a caller-owned device buffer the library copies
 * into (on the stream, after the estimation).  s = m/2 + 1 solved samples per
 * direction (samples m - j are the conjugates of samples j); complex values
 * are (re, im) pairs.
 *   p_z2[k]: double complex [n][c][s][H_Bk]  samples of B_k at z2 = w^j (Eq. 3)
 *   p_z1[k]: double complex [n][c][s][W_Bk]  samples of B_k at z1 = w^i
 *   x_z2, x_z1: double complex [n][s][t1+t2] unit null vectors [u; v] per sample
 *   sample_diag: double [n][2][s][4]: lambda_max, second smallest eigenvalue and
 *            Rayleigh quotient of the per-sample normal matrix, 1 if solved by
 *            the double-precision block inverse iteration
 *   lifted:  double complex [n][4][m][m]: A_1, A_2 (z2-first order), B_1, B_2
 *            (z1-first order) estimates of the kernels' m x m DFT
 *   kernels: double [n][t1*t1 + t2*t2]: K1 then K2 before the dtype cast */
typedef struct cbp_stage_out {
  void* p_z2[2];
  void* p_z1[2];
  void* x_z2;
  void* x_z1;
  void* sample_diag;
  void* lifted;
  void* kernels;
} cbp_stage_out;

/* cbp_estimate_kernels plus copies of the intermediates into `out` (may be NULL). */
cbp_status cbp_estimate_kernels_stages(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                                       const cbp_params* params, void* k1, void* k2,
                                       cbp_diag* diag, const cbp_stage_out* out, void* stream);

/* cbp_estimate_kernels without any device allocation and without a context.
 * The paper has no counterpart: this serves callers that may not allocate
 * device memory -- code under a memory manager that owns every allocation,
 * real-time paths that must not fail on an allocation, deployments that keep
 * a fixed device footprint.  The workspace is a fixed 16 MiB device array in
 * the library (held by every GPU that loads it until the process exits);
 * problems whose estimation workspace (cbp_workspace_size without the
 * deconvolution buffers) exceeds it return CBP_ERR_UNSUPPORTED -- one
 * 1080p RGB pair with 15x15 and 17x17 kernels fits on either path (7.1 MB
 * FP64, 9.7 MB mixed), three do not.  Inputs and outputs are as in cbp_estimate_kernels (device buffers;
 * CBP_FLAG_HOST_IO and CBP_FLAG_KERNELS_IN are rejected with
 * CBP_ERR_INVALID_ARG; the learned path with CBP_ERR_UNSUPPORTED).
 * The array's address is looked up with the caller's device current on every
 * call made outside stream capture and remembered per device and context; a
 * call made while its stream is capturing uses the remembered address, so
 * make the first call on a device (and the first after a device reset) before
 * any stream capture.  Every call shares the array and finds the previous
 * call's data in it; calls that overlap on the GPU race on it, so the caller
 * must order them (one stream, or synchronise). */
cbp_status cbp_estimate_kernels_noalloc(const cbp_frames* b1, const cbp_frames* b2,
                                        const cbp_params* params, void* k1, void* k2,
                                        cbp_diag* diag, void* stream);

/* Kernel estimation (as above, unless CBP_FLAG_KERNELS_IN) followed by the
 * dual-kernel Fourier deconvolution on a pad_h x pad_w grid:
 *   I^ = (conj(K1^) B1^ + conj(K2^) B2^) / (|K1^|^2 + |K2^|^2 + eps),
 * latent = real(IDFT(I^))[0:H, 0:W] per channel (Section 4 divides B1 by K1
 * in the Fourier domain; CBP_FLAG_SINGLE_KERNEL selects that form,
 * conj(K1^) B1^ / (|K1^|^2 + eps)).
 * k1, k2: NULL (kernels kept internal) or device buffers as in
 * cbp_estimate_kernels (inputs with CBP_FLAG_KERNELS_IN).
 * latent: device, n * c * H * W elements of b1's dtype, contiguous.
 * With CBP_FLAG_HOST_IO every buffer is a host buffer and the copies are part
 * of the call.  Errors as cbp_estimate_kernels. */
cbp_status cbp_deblur_pair(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                           const cbp_params* params, void* k1, void* k2, void* latent,
                           cbp_diag* diag, void* stream);

/* Forward model of Eq. 1 (the camera side of Section 3): out = L (x) K + N,
 * full 2D convolution of every channel of a latent batch with one kernel per
 * batch entry, plus N(0, sigma^2) noise from a counter-based generator
 * (Philox-4x32-10) keyed by `seed` (sigma = 0: no noise).
 * latent: device, n x c x h x w of dtype; kernel: device, n x t x t doubles;
 * out: device, n x c x (h + t - 1) x (w + t - 1) of dtype, contiguous. */
cbp_status cbp_forward_blur(cbp_ctx* ctx, const void* latent, int32_t n, int32_t c,
                            int32_t h, int32_t w, cbp_dtype dtype, const double* kernel,
                            int32_t t, double sigma, uint64_t seed, void* out, void* stream);

/* Camera side of the scheme (Section 3, "Blur Kernel Selection" and the
 * cascaded pair). */
typedef struct cbp_encrypt_params {
  int32_t t1, t2;       /* sizes of the pair's kernels (public K1, private K2), 1..32    */
  int32_t t3, t4;       /* sizes of the cascade's pair (0, 0: no cascade)                */
  int32_t m;            /* samples per direction of the coprimality test; 0 => max of
                           the pair's sizes (the deblurring's default M), <= 32         */
  int32_t max_attempts; /* draws per frame and pair before giving up; 0 => 8           */
  double tol;           /* coprime when every sample's sigma_min / sigma_max > tol;
                           0 => 1e-7                                                     */
  double sigma;         /* sensor noise N(0, sigma^2) on both streams (not the cascade)  */
  uint64_t seed;        /* key of the generator                                          */
  int32_t frame0;       /* frame index of the batch's first frame (generator counter)    */
  int32_t reserved;
} cbp_encrypt_params;

/* Encrypt a batch of latent frames on the device (Section 3): for every frame
 * f a new pair of random square kernels -- entries uniform in (0, 1] from
 * Philox-4x32-10 (entry e of kernel `kind` at redraw a: word e mod 4 of
 * Philox(counter = (e / 4, frame0 + f, 256 kind + a, 0), key = seed), value
 * (word + 1) 2^-32), normalised to unit sum -- redrawn until the pair passes
 * the coprimality test: at every sample w^j (w = exp(-2 pi i / m)) of both
 * evaluation orders the univariate kernel polynomials share no root
 * (sigma_min / sigma_max of their Sylvester matrix > tol) and one keeps full
 * degree.  Then B1 = L (x) K1 + N1 (public stream) and B2 = L (x) K2 + N2
 * (private stream), full 2D convolution per channel (Eq. 1).  With a cascade
 * (t3, t4 > 0), a second coprime pair (kinds 2, 3) blurs the public stream
 * again: C1 = B1 (x) K3, C2 = B1 (x) K4, the pair distributed where the
 * first pair's private stream may not go.
 * latent: device, n x c x h x w of dtype.  k1, k2 (k3, k4): device, n t_k^2
 * doubles.  b1, b2: device, n x c x (h + t_k - 1) x (w + t_k - 1) of dtype.
 * c1, c2: NULL without a cascade, else n x c x (h + t1 + t3 - 2) x
 * (w + t1 + t3 - 2) and (... t4 ...).  attempts: NULL or host array of n
 * (2 n with a cascade: the cascade's after the pair's) accepted draw indices,
 * -1 where every draw failed (the last draw is used).  The draws synchronise
 * the stream once per redraw round (usually one round).
 * Errors: CBP_ERR_INVALID_ARG, CBP_ERR_BUDGET, CBP_ERR_OOM, CBP_ERR_CUDA. */
cbp_status cbp_encrypt(cbp_ctx* ctx, const void* latent, int32_t n, int32_t c, int32_t h, int32_t w,
                       cbp_dtype dtype, const cbp_encrypt_params* params, double* k1, double* k2,
                       void* b1, void* b2, double* k3, double* k4, void* c1, void* c2,
                       int32_t* attempts, void* stream);

/* Multi-level security (Section 3): the private stream as a lower clearance
 * level receives it, with the least significant bits of its pixel codes
 * removed.  Each of the `count` elements x (intensities nominally in [0, 1])
 * is coded as code = rint(x (2^bits - 1)) clamped to [0, 2^bits - 1]; the
 * `drop` lowest bits of the code are cleared and the value
 * code / (2^bits - 1) written to out (same dtype; out may equal in).  The
 * arithmetic is double precision for either dtype.  in, out: device buffers.
 * Errors: CBP_ERR_INVALID_ARG (1 <= bits <= 30, 0 <= drop < bits),
 * CBP_ERR_CUDA. */
cbp_status cbp_truncate_lsb(cbp_ctx* ctx, const void* in, cbp_dtype dtype, int64_t count,
                            int32_t bits, int32_t drop, void* out, void* stream);

/* Bounds-checked builds (the library compiled with -DCBP_CHECKS: the
 * diagnostic variant libcbp_checks.so; the paper has no counterpart).  The
 * kernels check the indices of their main global stores and shared-memory
 * staging; a failed check sets a bit in its source file's check word and
 * skips the access instead of faulting.  Waits for the device, then writes n
 * words (word i: one source file, bit b: one checked site, 0 = no failure)
 * and clears them if reset != 0.  Host buffer.
 * Errors: CBP_ERR_UNSUPPORTED (a normal build), CBP_ERR_INVALID_ARG,
 * CBP_ERR_CUDA. */
cbp_status cbp_check_words(uint32_t* words, int32_t n, int32_t reset);

/* Checked builds only: with on != 0 every bulk-copy barrier of the row passes
 * expects 16 bytes more than its copies deliver, so the copies all land but no
 * phase completes and each bounded wait runs out; a call then reports
 * CBP_ERR_TIMEOUT in every pair's diagnostics, with no copy in flight and the
 * context still usable.  For testing the timeout path; on = 0 restores normal
 * operation.  Waits for the device first.
 * Errors: CBP_ERR_UNSUPPORTED (a normal build), CBP_ERR_CUDA. */
cbp_status cbp_check_expire_waits(int32_t on);

/* Verification of the solver's double-precision reciprocal and reciprocal
 * square root (the paper has no counterpart): the Newton-Raphson iteration
 * from a single-precision seed, two steps, used inside the eigen-solver for
 * 1e-30 < |x| < 1e30 (plain division and sqrt outside).  For each of the n
 * device doubles x: rcp = 1 / x, rsqrt = 1 / sqrt(x) (0 where x <= 0), as the
 * solver computes them.  Device buffers; no context.
 * Errors: CBP_ERR_INVALID_ARG, CBP_ERR_CUDA. */
cbp_status cbp_check_recip(const double* x, int64_t n, double* rcp, double* rsqrt, void* stream);

/* Synthetic latent frames for benchmarks (stand-in for the paper's camera
 * video, Section 6): for every channel, sum of Gaussian blobs
 * a * exp(-((x-cx)^2 + (y-cy)^2) / (2 s^2)) plus a uniform floor U[0, floor_amp]
 * from Philox-4x32-10 keyed by `seed`.
 * blobs: device, n x c x nblobs x 4 doubles (a, s, cx, cy); out: device,
 * n x c x h x w of dtype, contiguous. */
cbp_status cbp_synth_latent(cbp_ctx* ctx, const double* blobs, int32_t nblobs, int32_t n,
                            int32_t c, int32_t h, int32_t w, cbp_dtype dtype, double floor_amp,
                            uint64_t seed, void* out, void* stream);

/* Per-stage timing (the paper's Table 1 reports per-stage times, Section 6).
 * With profiling enabled, every call on the context brackets each stage with
 * CUDA events on its stream; cbp_stage_times() waits for the recorded events,
 * adds each stage's elapsed milliseconds into ms[stage] and its kernel-launch
 * count into launches[stage] (arrays of CBP_NUM_STAGES entries, either may be
 * NULL), and clears the record.  Stages of the serving engine are not timed. */
typedef enum cbp_stage {
  CBP_STAGE_EVAL = 0,           /* A1: fold bins -> samples (deblur: 1 kernel;
                                   estimate only: fold row pass + bins, 2)       */
  CBP_STAGE_SAMPLE_SOLVE = 1,   /* A2-A3: per-sample Gram + null vector          */
  CBP_STAGE_SCALE_SOLVE = 2,    /* A4-A5: lift, scale fix, inverse DFT           */
  CBP_STAGE_KERNEL_SPECTRA = 3, /* kernels' spectra on the FFT grid (+ twiddles) */
  CBP_STAGE_ROW_FFT = 4,        /* one read of B1, B2: A1 folds + forward real
                                   row FFTs                                      */
  CBP_STAGE_COL_DECONV = 5,     /* column FFTs + dual-kernel formula + inverse    */
  CBP_STAGE_ROW_IFFT = 6,       /* inverse row FFTs, crop, scale                  */
  CBP_STAGE_H2D = 7,            /* host-to-device copies (CBP_FLAG_HOST_IO)       */
  CBP_STAGE_D2H = 8,            /* device-to-host copies (CBP_FLAG_HOST_IO)       */
  CBP_STAGE_PROPOSAL = 9,       /* learned path: network proposal                */
  CBP_STAGE_GATE = 10,          /* learned path: proposal spectra + residual gate */
  CBP_NUM_STAGES = 11
} cbp_stage;

cbp_status cbp_profile(cbp_ctx* ctx, int32_t enable);
cbp_status cbp_stage_times(cbp_ctx* ctx, double* ms, int64_t* launches);

/* --- serving: continuous batching of independent requests (frame pairs of
 * any supported shape).  cbp_stream_submit copies the request descriptor and
 * returns at once with a ticket; a scheduler thread admits requests when a
 * workspace slot and HBM budget are free, batches requests of the same shape
 * bucket, and runs them on a pool of streams with captured CUDA graphs.
 * Buffers are device buffers owned by the caller and must stay valid until
 * the request completes.  Thread-safe. ---------------------------------- */
cbp_status cbp_stream_submit(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                             const cbp_params* params, void* k1, void* k2, void* latent,
                             uint64_t* ticket);

/* Wait up to timeout_us (0: do not wait, < 0: wait without limit) for a
 * ticket.  Returns the request's status once done (diag filled if non-NULL;
 * the ticket is then released), CBP_ERR_BUSY if not done yet and
 * timeout_us == 0, CBP_ERR_TIMEOUT if the limit passed,
 * CBP_ERR_INVALID_ARG for an unknown ticket. */
cbp_status cbp_stream_poll(cbp_ctx* ctx, uint64_t ticket, int32_t timeout_us, cbp_diag* diag);

/* Serving statistics: completed requests, p50 and p99 latency (ms, submit to
 * completion) since the last reset; reset when `reset` != 0. */
cbp_status cbp_stream_stats(cbp_ctx* ctx, uint64_t* completed, double* p50_ms,
                            double* p99_ms, int32_t reset);

/* --- learned kernel proposal (CBP_PATH_LEARNED) --------------------------
 * A small network proposes both kernels from the two blurred frames (an
 * addition to the paper, whose kernels come only from the GCD solve of
 * Sections 4-5): the luma (channel mean) of each frame, area-downsampled to
 * 256 x 256, then conv 3x3 stride 2 pad 1 (2 -> 32) + ReLU, conv 3x3 stride 2
 * pad 1 (32 -> 32) + ReLU, conv 3x3 stride 4 pad 1 (32 -> 32) + ReLU,
 * conv 2x2 (32 -> 2), softmax over each channel's 15 x 15 logits: K1, K2.
 * Activations bfloat16, weights kept in float32 (rounded to bfloat16 for the
 * tensor-core products), accumulation float32.  A weight vector is
 * cbp_cnn_param_count() floats: w1 [32][2][3][3], b1 [32], w2 [32][32][3][3],
 * b2 [32], w3 [32][32][3][3], b3 [32], w4 [2][32][2][2], b4 [2].
 *
 * With params->path == CBP_PATH_LEARNED (t1 == t2 == 15, weights loaded by
 * cbp_learned_load) cbp_deblur_pair runs the network, computes the
 * consistency residual rho = ||B1*K2 - B2*K1|| / ||B1|| of the proposal
 * (circular convolutions on the deconvolution grid, via Parseval) and keeps
 * the proposal where rho <= accept_rho; the other pairs take the mixed
 * GCD solve.  diag.rho and diag.used_fallback report the decision. */
typedef struct cbp_cnn_trace {   /* optional device float32 copies; NULL skips */
  float* input;    /* [n][2][256][256] network input                          */
  float* act[3];   /* [n][32][128][128], [n][32][64][64], [n][32][16][16]     */
  float* logits;   /* [n][2][15][15]                                          */
  float* grad;     /* [param count] batch-loss gradient (training step only)   */
} cbp_cnn_trace;

typedef struct cbp_adamw {
  float lr, beta1, beta2, eps, weight_decay;  /* decoupled weight decay      */
  int32_t step;                                 /* 1 for the first step       */
} cbp_adamw;

size_t cbp_cnn_param_count(void);

/* Proposals for n pairs: kernels = device float32 [n][2][15][15] (K1, K2).
 * weights: device float32 vector, or NULL for the context's loaded weights;
 * the convolutions run on the tensor cores with the weights rounded to
 * bfloat16 and bfloat16 activations, accumulating in float32 (a tensor-core
 * completion that does not arrive in time leaves NaN proposals).
 * Frames as for cbp_estimate_kernels (any size; both of one dtype).  Async. */
cbp_status cbp_cnn_forward(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                           const float* weights, float* kernels, cbp_cnn_trace* trace,
                           void* stream);

/* One training step on n pairs: loss = mean over pairs and entries of
 * (K - k_true)^2, k_true device float32 [n][2][15][15]; backward pass (its
 * products on the tensor cores with bfloat16 operands and float32
 * accumulation, the bias gradients summed in float32, every reduction in a
 * fixed order), then AdamW on the device float32 weights with moments
 * adam_m, adam_v (same length, zero before the first step).  loss: device
 * float32 [1] or NULL. */
cbp_status cbp_cnn_train_step(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                              const float* k_true, float* weights, float* adam_m, float* adam_v,
                              const cbp_adamw* hp, float* loss, cbp_cnn_trace* trace,
                              void* stream);

/* Load weights for CBP_PATH_LEARNED from a file: 8 bytes "CBPCNN1\0", int32
 * side (256), int32 count (cbp_cnn_param_count()), count float32 values,
 * little-endian.  Synchronous. */
cbp_status cbp_learned_load(cbp_ctx* ctx, const char* weights_path);

#ifdef __cplusplus
}
#endif
#endif /* CBP_H_ */
