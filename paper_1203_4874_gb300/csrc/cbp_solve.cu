// A2-A5: per-sample cofactor solve, scale fix between the two evaluation
// orders, and the spatial kernels (Eq. 4; Sections 4-5).
//
// Per sample: the 1D cofactor pair x = [u; v] (u ~ k1, v ~ k2
// at that sample) spans the null space of the Sylvester matrix
// S = [-C_t1(b2) | C_t2(b1)], channels' rows stacked, since b1 k2 - b2 k1 = 0
// (Eq. 4).  The paper factors Bezout matrices by a CPU SVD (Section 5); here
// the normal matrix G = S^H S is formed on the device from correlations --
// its blocks are Toeplitz, (C_t(a)^H C_s(b))[p][q] = rho_ab(p - q) with
// rho_ab(d) = sum_m conj(a[m]) b[m + d] -- by one CTA per sample
// (k_sample_gram), and its smallest eigenvector is found by one warp per
// sample (k_sample_solve, cbp_tri.cuh):
//   1. Householder reduction to a real tridiagonal T in double precision;
//   2. Sturm-count multisection for the two smallest eigenvalues of T;
//   3. inverse iteration on T, x = Q y;
//   4. Newton steps (Olsen's form, solved through T) whose residual S^H S x
//      is computed from S itself (convolutions), which removes the squared
//      conditioning of the normal matrix: FP64 path always, mixed path where
//      the two smallest eigenvalues are nearly degenerate (the z = 1
//      samples, whose lower spectrum is a cluster of noise-level eigenvalues).
// Only samples s <= M/2 are solved; sample M - s is the conjugate.
//
// Per pair (one CTA): lift the cofactors to the two M x M estimates of the
// kernels' 2D DFT, solve the least-squares scale system (the tridiagonal
// eigen-solver on its 2M x 2M normal matrix, one exact-residual step on the
// FP64 path), average,
// normalise to unit kernel sum, inverse M x M DFT (Section 5).
#include <algorithm>
#include "cbp_common.cuh"
#include "cbp_ff.cuh"
#include "cbp_internal.h"
#if defined(CBP_PHASE_TIMING) || defined(CBP_SCHED_TRACE)
#include <cstdio>
#endif

namespace cbp {

CBP_CHECKS_TU(kChkSolve)

namespace {

constexpr int kSolveThreads = 256;
#ifndef CBP_SOLVE_WPC
#define CBP_SOLVE_WPC 4
#endif

// Optional per-phase cycle counts (build with -DCBP_PHASE_TIMING): thread 0 of
// a few blocks prints the clock64 deltas between the solver's phases.
#ifdef CBP_PHASE_TIMING
#define CBP_TICK(arr, i) \
  do {                   \
    if (threadIdx.x == 0) (arr)[i] = clock64(); \
  } while (0)
#else
#define CBP_TICK(arr, i) \
  do {                   \
  } while (0)
#endif

// ------------------------------------------------------------ block helpers
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// Scalar helpers so one solver serves real (float, double) and complex data.
__device__ __forceinline__ float re_(float x) { return x; }
__device__ __forceinline__ double re_(double x) { return x; }
template <typename T> __device__ __forceinline__ T re_(cpx<T> x) { return x.re; }
__device__ __forceinline__ float cj_(float x) { return x; }
__device__ __forceinline__ double cj_(double x) { return x; }
template <typename T> __device__ __forceinline__ cpx<T> cj_(cpx<T> x) { return conj(x); }
__device__ __forceinline__ float a2_(float x) { return x * x; }
__device__ __forceinline__ double a2_(double x) { return x * x; }
template <typename T> __device__ __forceinline__ T a2_(cpx<T> x) { return abs2(x); }
__device__ __forceinline__ double warp_sum_e(double v) { return warp_sum(v); }
__device__ __forceinline__ cd warp_sum_e(cd v) { return mk(warp_sum(v.re), warp_sum(v.im)); }
template <typename E> struct Ops;
template <> struct Ops<double> {
  static __device__ double z() { return 0.0; }
  static __device__ double o() { return 1.0; }
  static __device__ void clear_im(double&) {}
  static __device__ bool nz(double x) { return x != 0.0; }
};
template <typename T> struct Ops<cpx<T>> {
  static __device__ cpx<T> z() { return mk<T>((T)0, (T)0); }
  static __device__ cpx<T> o() { return mk<T>((T)1, (T)0); }
  static __device__ void clear_im(cpx<T>& x) { x.im = (T)0; }
  static __device__ bool nz(cpx<T> x) { return x.re != (T)0 || x.im != (T)0; }
};

// Reciprocal and reciprocal square root in double precision by the
// Newton-Raphson iteration: a single-precision seed (relative error below
// 2^-23) refined by two Newton steps for f(y) = 1/y - x, y <- y (2 - x y), and
// for f(y) = 1/y^2 - x, y <- y (3 - x y^2) / 2; each step squares the
// relative error, so two take it below double rounding.  Valid for x within
// the float range (callers guard 1e-30 < |x| < 1e30).  Cheap on a GPU whose
// double pipe is slow; cbp_check_recip exposes them for verification.
__device__ __forceinline__ double rcp_d(double x) {
  double y = (double)(1.0f / (float)x);
  y = y * fma(-x, y, 2.0);
  return y * fma(-x, y, 2.0);
}
__device__ __forceinline__ double rsqrt_d(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x * y, y, 1.5);
  return y * fma(-0.5 * x * y, y, 1.5);
}
__device__ __forceinline__ float rcp_d(float x) { return 1.0f / x; }
__device__ __forceinline__ float rsqrt_d(float x) { return rsqrtf(x); }

__device__ __forceinline__ void fma_(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void fma_(cd& acc, cd a, cd b) { cfma(acc, a, b); }
__device__ __forceinline__ cd to_cd(double v) { return mk(v, 0.0); }
__device__ __forceinline__ cd to_cd(cd v) { return v; }

// ------------------------------------------------------ per-sample solve ---
struct SampleArgs {
  const cd* pz[2][2];        // [pass][frame] double samples [n][C][ns][len]
  const cdf* pzf[2][2];      // [pass][frame] float-float copies (mixed path), same layout
  int len[2][2];             // [pass][frame]
  cd* X;                     // [n][2][ns][nn]
  double* sdiag;             // [n][2][ns][4]
  cd* resid;                 // [n][2][ns][C][Lmax]
  const int* accepted;       // learned path: pairs whose proposal passed the gate (skipped)
  cd* G;                     // [n][2][ns][nn][nn] normal matrices
  int Lmax, C, ns, t1, t2, nn, M, mixed;
  int nfr;                   // pairs in the call
};

// Sample polynomial element m of frame k (0: b1, 1: b2) as cpx<TA>.
template <typename TP, typename TA>
struct SamplePolys {
  const cpx<TP>* c[2];   // channel 0 of the sample; channel stride cstride[k]
  int64_t cstride[2];
  int len[2];
  __device__ __forceinline__ cpx<TA> ld(int k, int ch, int m) const {
    cpx<TP> v = c[k][ch * cstride[k] + m];
    return mk<TA>((TA)v.re, (TA)v.im);
  }
};

template <typename TP, typename TA>
__device__ SamplePolys<TP, TA> sample_polys(const cpx<TP>* const base[2], const int len[2], int f,
                                            int C, int ns, int s) {
  SamplePolys<TP, TA> P;
  for (int k = 0; k < 2; ++k) {
    P.len[k] = len[k];
    P.c[k] = base[k] + ((int64_t)f * C * ns + s) * len[k];
    P.cstride[k] = (int64_t)len[k] * ns;
  }
  return P;
}

// rho jobs: j < t1: rho_22(j); j < t1+t2: rho_11(j - t1);
// else rho_21(d), d = j - t1 - t2 - (t2 - 1) in [-(t2-1), t1-1].
template <typename TP, typename TA>
__device__ void correlations(const SamplePolys<TP, TA>& P, int C, int t1, int t2, cd* rho) {
  const int J = 2 * (t1 + t2) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < J; j += nw) {
    int ka, kb, d;
    if (j < t1) { ka = 1; kb = 1; d = j; }
    else if (j < t1 + t2) { ka = 0; kb = 0; d = j - t1; }
    else { ka = 1; kb = 0; d = j - t1 - t2 - (t2 - 1); }
    const int la = P.len[ka], lb = P.len[kb];
    const int m0 = d < 0 ? -d : 0;
    const int m1 = min(la, lb - d);
    cpx<TA> acc = mk<TA>(0, 0);
    for (int ch = 0; ch < C; ++ch)
      for (int m = m0 + lane; m < m1; m += 32) cfmac(acc, P.ld(ka, ch, m), P.ld(kb, ch, m + d));
    double re = warp_sum((double)acc.re), im = warp_sum((double)acc.im);
    if (lane == 0) rho[j] = mk(re, im);
  }
  __syncthreads();
}

// rho jobs as above for real samples (z = 1, and z = -1 when M is even):
// real double correlations of the real parts.
__device__ void correlations_real(const SamplePolys<double, double>& P, int C, int t1, int t2,
                                  cd* rho) {
  const int J = 2 * (t1 + t2) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j < J; j += nw) {
    int ka, kb, d;
    if (j < t1) { ka = 1; kb = 1; d = j; }
    else if (j < t1 + t2) { ka = 0; kb = 0; d = j - t1; }
    else { ka = 1; kb = 0; d = j - t1 - t2 - (t2 - 1); }
    const int la = P.len[ka], lb = P.len[kb];
    const int m0 = d < 0 ? -d : 0;
    const int m1 = min(la, lb - d);
    double acc = 0;
    for (int ch = 0; ch < C; ++ch) {
      const cd* a = P.c[ka] + ch * P.cstride[ka];
      const cd* b = P.c[kb] + ch * P.cstride[kb];
      for (int m = m0 + lane; m < m1; m += 32) acc = fma(a[m].re, b[m + d].re, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) rho[j] = mk(acc, 0.0);
  }
  __syncthreads();
}

// Float-float accumulation (hi + lo) on the single-precision units.
struct FF {
  float hi = 0.f, lo = 0.f;
  // += a * b for float-float a, b: exact product of the high parts (FMA) plus
  // the cross terms; the high part by TwoSum, every rounding term into lo
  // (renormalised only when sums are combined: over a lane's ~100 terms lo
  // stays ~1e-13 of the diagonal of the normal matrix).
  __device__ __forceinline__ void mac(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    const float t = hi + p;
    const float z = t - hi;
    lo += ((hi - (t - z)) + (p - z)) + e;
    hi = t;
  }
  __device__ __forceinline__ void add(float bh, float bl) {
    const float t = hi + bh;
    const float z = t - hi;
    const float err = (hi - (t - z)) + (bh - z);
    const float l = lo + err + bl;
    hi = t + l;
    lo = l - (hi - t);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_xor_sync(0xffffffffu, v.hi, o);
    const float l = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v.add(h, l);
  }
  return v;
}

// rho jobs as above from float-float samples: conj(a) b accumulated in
// float-float, about 1e-13 relative, on the single-precision units.  The
// samples pass through shared memory in tiles of kGramChunk positions (plus a
// halo of kMaxN each side, zero outside the polynomials, so every product
// outside a lag's overlap is an exact zero); warp w takes the lags
// j = w, w + 8, ..., a lane the positions lane + 32 r of each tile.  The next
// tile's loads are in flight while the current one is summed.
constexpr int kGramChunk = 256;
constexpr int kGramTile = kGramChunk + 2 * kMaxN;
constexpr int kGramLags = 8;     // lags per warp and pass
constexpr int kGramPre = (2 * kGramTile + kSolveThreads - 1) / kSolveThreads;

__device__ void correlations_ff(const cdf* const base[2], const int len[2], int f, int C, int ns,
                                int s, int t1, int t2, cd* rho, cdf* tile /* [2][kGramTile] */) {
  const int J = 2 * (t1 + t2) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int maxlen = max(len[0], len[1]);
  const int nchunk = (maxlen + kGramChunk - 1) / kGramChunk;
  const int iters = C * nchunk;
  const cdf zero = {0.f, 0.f, 0.f, 0.f};
  auto fetch = [&](int it, cdf* pre) {
    const int ch = it / nchunk, m0 = (it - ch * nchunk) * kGramChunk - kMaxN;
#pragma unroll
    for (int q = 0; q < kGramPre; ++q) {
      const int e = threadIdx.x + q * kSolveThreads;
      const int k = e / kGramTile, g = m0 + (e - k * kGramTile);
      pre[q] = zero;
      if (e < 2 * kGramTile && g >= 0 && g < len[k])
        pre[q] = base[k][((int64_t)(f * C + ch) * ns + s) * len[k] + g];
    }
  };
  for (int j0 = 0; j0 < J; j0 += kGramLags * nw) {     // passes over the lags
    FF re[kGramLags], im[kGramLags];
    cdf pre[kGramPre];
    fetch(0, pre);
    for (int it = 0; it < iters; ++it) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kGramPre; ++q) {
        const int e = threadIdx.x + q * kSolveThreads;
        if (e < 2 * kGramTile) tile[e] = pre[q];
      }
      __syncthreads();
      if (it + 1 < iters) fetch(it + 1, pre);
#pragma unroll
      for (int q = 0; q < kGramLags; ++q) {
        const int j = j0 + warp + q * nw;
        if (j >= J) break;
        int ka, kb, d;
        if (j < t1) { ka = 1; kb = 1; d = j; }
        else if (j < t1 + t2) { ka = 0; kb = 0; d = j - t1; }
        else { ka = 1; kb = 0; d = j - t1 - t2 - (t2 - 1); }
        const cdf* A = tile + ka * kGramTile + kMaxN;
        const cdf* B = tile + kb * kGramTile + kMaxN + d;
#pragma unroll 4
        for (int r = 0; r < kGramChunk / 32; ++r) {
          const int m = lane + 32 * r;
          const cdf x = A[m], y = B[m];
          // conj(x) y = (xr yr + xi yi) + i (xr yi - xi yr)
          re[q].mac(x.rh, x.rl, y.rh, y.rl);
          re[q].mac(x.ih, x.il, y.ih, y.il);
          im[q].mac(x.rh, x.rl, y.ih, y.il);
          im[q].mac(-x.ih, -x.il, y.rh, y.rl);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kGramLags; ++q) {
      const int j = j0 + warp + q * nw;
      const FF sr = warp_sum_ff(re[q]), si = warp_sum_ff(im[q]);
      if (j < J && lane == 0) rho[j] = mk(sr.value(), si.value());
    }
  }
  __syncthreads();
}

// G[p][q] from the correlations (Toeplitz blocks).
__device__ void gram_from_rho(const cd* rho, int t1, int t2, cd* G) {
  const int n = t1 + t2;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    int p = i / n, q = i % n;
    cd g;
    if (p < t1 && q < t1) {
      int d = p - q;
      g = d >= 0 ? rho[d] : conj(rho[-d]);
    } else if (p >= t1 && q >= t1) {
      int d = (p - t1) - (q - t1);
      g = d >= 0 ? rho[t1 + d] : conj(rho[t1 - d]);
    } else if (p < t1) {
      int d = p - (q - t1);               // rho_21(d)
      cd v = rho[t1 + t2 + d + t2 - 1];
      g = mk(-v.re, -v.im);
    } else {
      int d = q - (p - t1);
      cd v = rho[t1 + t2 + d + t2 - 1];
      g = mk(-v.re, v.im);                // -conj(rho_21(d))
    }
    G[i] = g;
  }
  __syncthreads();
}

// Accurate S^H S x for the FP64 path: y = S x per channel in the global
// scratch, then the correlations with b1, b2.
#include "cbp_tri.cuh"

// S^H S x from the double samples (the exact operator of the refinement
// steps; y holds S x), by the whole CTA (BLOCK) or by the calling warp.
// S = [-C_t1(b2) | C_t2(b1)] (channels' rows stacked):
//   (S x)[ch][i] = sum_q b1[ch][i - q] v_q - sum_p b2[ch][i - p] u_p,
//   (S^H y)_u[p] = -sum_ch sum_m conj(b2[ch][m]) y[ch][m + p], likewise v with b1.
template <bool BLOCK>
struct SylvesterApply {
  SamplePolys<double, double> P;
  const cdf* F[2];  // float-float samples (mixed path, complex samples) or null: read instead of P
  int64_t fstride[2];
  cd* y;            // [C][L]
  int C, t1, t2, L;
  bool real;        // real sample (z = 1, or z = -1 for even M): real arithmetic
  // float-float real samples: shared scratch of ys_cap float pairs (a
  // channel's S x and both polynomials when they fit, else y and the samples
  // are used in place), the warps' partial sums of S^H y in part[nw][n]
  float2* ys = nullptr;
  int ys_cap = 0;
  float2* part = nullptr;
  __device__ void operator()(const cd* x, cd* out) const {
    if (real) {
      if constexpr (BLOCK) {
        if (F[0]) {
          run_ff_real(x, out);
          return;
        }
      }
      run<true, false>(x, out);
    } else if (F[0]) {
      run<false, true>(x, out);
    } else {
      run<false, false>(x, out);
    }
  }
  // A real sample from float-float samples (mixed path), by the whole CTA:
  // the same two products in float-float arithmetic on the single-precision
  // units (each product exact to ~1e-14, rounding terms gathered in the low
  // part and renormalised at most every 32 terms), y held as float pairs.
  // Against the double products the double-precision units (a few per SM)
  // took, the single-precision ones take ~10 operations per product at 64
  // times the rate.  One channel at a time, its two polynomials staged in
  // shared memory; both products keep several independent sums per thread
  // (eight outputs of S x, four slices of each output of S^H y), so the
  // chains' latencies overlap instead of adding up.
  __device__ void run_ff_real(const cd* x, cd* out) const {
    __shared__ float2 xf[kMaxN];
    constexpr int R = 8;                       // outputs of S x per thread and pass
    const int lane = threadIdx.x & 31, nth = blockDim.x;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int len0 = P.len[0], len1 = P.len[1], n = t1 + t2;
    // one channel at a time: both polynomials (hi, lo) and that channel's S x
    // in shared memory when they fit, else read and written in place
    const bool stage = ys && ys_cap >= L + len0 + len1;
    team_sync<BLOCK>();
    for (int i = threadIdx.x; i < n; i += nth) {
      const float h = (float)x[i].re;
      xf[i] = make_float2(h, (float)(x[i].re - (double)h));
    }
    const int mmax = max(len0, len1), chunk = (mmax + nw - 1) / nw;
    const int nblk = (L + R - 1) / R;
    FF tot[2];                                 // this lane's outputs o = lane, lane + 32
    for (int ch = 0; ch < C; ++ch) {
      const float2* g0 = reinterpret_cast<const float2*>(F[0] + ch * fstride[0]);   // b1
      const float2* g1 = reinterpret_cast<const float2*>(F[1] + ch * fstride[1]);   // b2
      const float2* pb[2] = {g0, g1};
      int bs = 2;                              // float2 per coefficient
      float2* yc = reinterpret_cast<float2*>(y) + ch * L;
      team_sync<BLOCK>();                      // the last channel's reads are done
      if (stage) {
        float2* s0 = ys + L;
        float2* s1 = s0 + len0;
        // asynchronous copies: every thread's loads in flight at once
        for (int i = threadIdx.x; i < len0 + len1; i += nth) {
          const float2* src = i < len0 ? g0 + 2 * i : g1 + 2 * (i - len0);
          const unsigned dst = (unsigned)__cvta_generic_to_shared(s0 + i);
          if (CBP_CHECK(L + i < ys_cap, 0))
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        pb[0] = s0;
        pb[1] = s1;
        bs = 1;
        yc = ys;
        team_sync<BLOCK>();
      }
      // y = S x: each thread R consecutive outputs, the coefficient window slid
      // by one per term (R independent sums)
      for (int bi = threadIdx.x; bi < nblk; bi += nth) {
        const int i0 = bi * R;
        FF acc[R];
        for (int k = 0; k < 2; ++k) {          // k = 0: b1 * v (t2 terms); k = 1: -b2 * u (t1 terms)
          const float2* r = pb[k];
          const int lk = k ? len1 : len0, nt = k ? t1 : t2, x0 = k ? 0 : t1;
          const float sg = k ? -1.f : 1.f;
          float2 w[R];                         // w[j] = b[i0 + j - q]
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int m = i0 + j;
            w[j] = (m < lk) ? r[bs * m] : make_float2(0.f, 0.f);
          }
          for (int q = 0; q < nt; ++q) {
            const float2 c = xf[x0 + q];
#pragma unroll
            for (int j = 0; j < R; ++j) acc[j].mac(sg * w[j].x, sg * w[j].y, c.x, c.y);
#pragma unroll
            for (int j = R - 1; j > 0; --j) w[j] = w[j - 1];
            const int m = i0 - q - 1;
            w[0] = (m >= 0 && m < lk) ? r[bs * m] : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          if (i0 + j < L) {
            acc[j].add(0.f, 0.f);
            yc[i0 + j] = make_float2(acc[j].hi, acc[j].lo);
          }
        }
      }
      team_sync<BLOCK>();
      // S^H y, this channel's terms: lane <-> output o, warp <-> a slice of
      // the terms; four sums per lane (renormalised every 16 terms)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (32 * c >= n) break;
        const int o = 32 * c + lane;
        const bool act = o < n;
        const int k = o < t1 ? 1 : 0;          // u rows use b2, v rows use b1
        const int sh = o < t1 ? o : o - t1;
        const int lk = act ? (k ? len1 : len0) : 0;
        const float2* rk = pb[k];
        const float2* yr = yc + sh;
        FF a0, a1, a2, a3;
        const int mb = wid * chunk, me = min(mb + chunk, lk);
        int m = mb;
        while (m + 4 <= me) {
          const int stop = min(me, m + 64);
          for (; m + 4 <= stop; m += 4) {
            const float2 b0 = rk[bs * m], b1 = rk[bs * (m + 1)], b2 = rk[bs * (m + 2)],
                         b3 = rk[bs * (m + 3)];
            const float2 y0 = yr[m], y1 = yr[m + 1], y2 = yr[m + 2], y3 = yr[m + 3];
            a0.mac(b0.x, b0.y, y0.x, y0.y);
            a1.mac(b1.x, b1.y, y1.x, y1.y);
            a2.mac(b2.x, b2.y, y2.x, y2.y);
            a3.mac(b3.x, b3.y, y3.x, y3.y);
          }
          a0.add(0.f, 0.f);
          a1.add(0.f, 0.f);
          a2.add(0.f, 0.f);
          a3.add(0.f, 0.f);
        }
        for (; m < me; ++m) {
          const float2 b = rk[bs * m], v = yr[m];
          a0.mac(b.x, b.y, v.x, v.y);
        }
        a0.add(0.f, 0.f);
        a0.add(a1.hi, a1.lo);
        a0.add(a2.hi, a2.lo);
        a0.add(a3.hi, a3.lo);
        tot[c].add(a0.hi, a0.lo);
      }
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int o = 32 * c + lane;
      if (o < n) part[wid * n + o] = make_float2(tot[c].hi, tot[c].lo);
    }
    team_sync<BLOCK>();
    for (int o = threadIdx.x; o < n; o += nth) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) {
        const float2 v = part[w * n + o];
        s += (double)v.x + (double)v.y;
      }
      out[o] = o < t1 ? mk(-s, 0.0) : mk(s, 0.0);
    }
    team_sync<BLOCK>();
  }
  template <bool FFS>
  __device__ __forceinline__ cd ld(const void* row, int m) const {
    if (FFS) {
      const cdf v = ((const cdf*)row)[m];
      return mk((double)v.rh + (double)v.rl, (double)v.ih + (double)v.il);
    }
    return ((const cd*)row)[m];
  }
  __device__ __forceinline__ const void* row(int k, int ch, bool ffs) const {
    if (ffs) return (const void*)((k ? F[1] : F[0]) + ch * (k ? fstride[1] : fstride[0]));
    return (const void*)((k ? P.c[1] : P.c[0]) + ch * (k ? P.cstride[1] : P.cstride[0]));
  }
  template <bool REAL, bool FFS>
  __device__ void run(const cd* x, cd* out) const {
    const int lane = threadIdx.x & 31;
    const int tid = BLOCK ? threadIdx.x : lane, nth = BLOCK ? blockDim.x : 32;
    const int wid = BLOCK ? threadIdx.x >> 5 : 0, nw = BLOCK ? blockDim.x >> 5 : 1;
    const int len0 = P.len[0], len1 = P.len[1];
    team_sync<BLOCK>();
    for (int idx = tid; idx < C * L; idx += nth) {
      const int ch = idx / L, i = idx - ch * L;
      const void* r0 = row(0, ch, FFS);
      const void* r1 = row(1, ch, FFS);
      cd acc = mk(0.0, 0.0);
      const int q0 = max(0, i - len0 + 1), q1 = min(t2 - 1, i);
      for (int q = q0; q <= q1; ++q) {     // b1 * v
        const cd b = ld<FFS>(r0, i - q);
        if (REAL) acc.re = fma(b.re, x[t1 + q].re, acc.re);
        else cfma(acc, b, x[t1 + q]);
      }
      const int p0 = max(0, i - len1 + 1), p1 = min(t1 - 1, i);
      for (int p = p0; p <= p1; ++p) {     // - b2 * u
        const cd b = ld<FFS>(r1, i - p);
        if (REAL) {
          acc.re = fma(-b.re, x[p].re, acc.re);
        } else {
          const cd u = x[p];
          acc.re -= b.re * u.re - b.im * u.im;
          acc.im -= b.re * u.im + b.im * u.re;
        }
      }
      y[idx] = acc;
    }
    team_sync<BLOCK>();
    const int n = t1 + t2;
    for (int o = wid; o < n; o += nw) {
      const int k = o < t1 ? 1 : 0;       // u rows use b2, v rows use b1
      const int sh = o < t1 ? o : o - t1;
      const int lk = k ? len1 : len0;
      cd acc = mk(0.0, 0.0);
      for (int ch = 0; ch < C; ++ch) {
        const void* rk = row(k, ch, FFS);
        const cd* yr = y + ch * L + sh;
        for (int m = lane; m < lk; m += 32) {
          const cd b = ld<FFS>(rk, m);
          if (REAL) acc.re = fma(b.re, yr[m].re, acc.re);
          else cfmac(acc, b, yr[m]);
        }
      }
      const double re = warp_sum(acc.re), im = REAL ? 0.0 : warp_sum(acc.im);
      if (lane == 0) out[o] = o < t1 ? mk(-re, -im) : mk(re, im);
    }
    team_sync<BLOCK>();
  }
};

// A2: per sample, the correlations and the Toeplitz-block normal matrix, into
// the global array of normal matrices.
__global__ void __launch_bounds__(kSolveThreads) k_sample_gram(SampleArgs a) {
  __shared__ cd rho[4 * kMaxN];
  __shared__ cdf tile[2 * kGramTile];
  const int f = blockIdx.x, ps = blockIdx.y, s = blockIdx.z;
  if (a.accepted && a.accepted[f]) return;   // the proposal stands; nothing to solve
  if (!CBP_CHECK(a.t1 + a.t2 <= kMaxN && s < a.ns && ps < 2, 1)) return;   // rho's size (whole block)
  // Real samples (z = 1; z = -1 when M is even) have real Gram matrices.
  const bool real = s == 0 || 2 * s == a.M;
  const SamplePolys<double, double> P64 =
      sample_polys<double, double>(a.pz[ps], a.len[ps], f, a.C, a.ns, s);
  if (real) correlations_real(P64, a.C, a.t1, a.t2, rho);
  else if (a.mixed) correlations_ff(a.pzf[ps], a.len[ps], f, a.C, a.ns, s, a.t1, a.t2, rho, tile);
  else correlations(P64, a.C, a.t1, a.t2, rho);
  const int64_t o = ((int64_t)f * 2 + ps) * a.ns + s;
  gram_from_rho(rho, a.t1, a.t2, a.G + o * a.nn * a.nn);
}

// A3: the null vector of every sample's normal matrix (tridiagonal
// reduction, Sturm multisection, inverse iteration, refinement steps against
// S^H S as configured below).  The first nreal CTAs take one real sample each
// (z = 1, and z = -1 for even M: their refinement, the costliest step, runs
// on the whole CTA); the others take one complex sample per warp.
__global__ void k_sample_solve(SampleArgs a, int nreal) {
  extern __shared__ __align__(16) char smem[];
#ifdef CBP_SCHED_TRACE
  unsigned long long t_start;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
#endif
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
  const int n = a.nn;
  const int nrs = (a.M % 2 == 0) ? 2 : 1, ncs = a.ns - nrs;   // real / complex samples per pass
  const bool real = (int)blockIdx.x < nreal;
  int f, ps, s;
  if (real) {
    const int r = blockIdx.x;
    f = r / (2 * nrs);
    ps = (r / nrs) & 1;
    s = (r % nrs) ? a.M / 2 : 0;
  } else {
    const int c = ((int)blockIdx.x - nreal) * wpc + warp;
    if (c >= a.nfr * 2 * ncs) return;          // whole warp leaves together
    f = c / (2 * ncs);
    ps = (c / ncs) & 1;
    s = 1 + c % ncs;
  }
  if (a.accepted && a.accepted[f]) return;   // the proposal stands; nothing to solve
  // a real sample's whole CTA, or a complex sample's warp, leaves together
  if (!CBP_CHECK(f < a.nfr && s < a.ns && n <= kMaxN, 2)) return;
  const int64_t o = ((int64_t)f * 2 + ps) * a.ns + s;
  const TriWs W = carve_tri(smem + (real ? 0 : (size_t)warp * tri_ws_bytes(n)), n);
  const cd* G = a.G + o * n * n;
#ifdef CBP_PHASE_TIMING
  long long tkv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long* tk = f == 0 ? tkv : nullptr;
#else
  long long* tk = nullptr;
#endif
  // Refinement against S^H S (it removes the squared conditioning of the
  // normal matrix; one step through T, accurate to double precision, takes x
  // to the double-precision floor).  FP64 path: one step.  Mixed path: one
  // step where the two smallest eigenvalues are within 1e-6 lambda_max (the
  // z = 1 samples: ~1e-9 apart, where the float-float normal matrix alone
  // leaves ~1e-4 in x), none elsewhere.
  const int far = a.mixed ? 0 : 1;
  const double gap = a.mixed ? 1e-6 : 1e-4;
  TriResult res;
  if (real) {
    SylvesterApply<true> ap;
    ap.P = sample_polys<double, double>(a.pz[ps], a.len[ps], f, a.C, a.ns, s);
    ap.C = a.C;
    ap.t1 = a.t1;
    ap.t2 = a.t2;
    ap.L = a.len[ps][0] + a.t2 - 1;
    ap.y = a.resid + o * a.C * (int64_t)a.Lmax;
    ap.F[0] = ap.F[1] = nullptr;
    if (a.mixed) {   // the refinement step in float-float arithmetic
      for (int k = 0; k < 2; ++k) {
        ap.F[k] = a.pzf[ps][k] + ((int64_t)f * a.C * a.ns + s) * a.len[ps][k];
        ap.fstride[k] = (int64_t)a.len[ps][k] * a.ns;
      }
    }
    ap.real = true;
    ap.part = reinterpret_cast<float2*>(W.part);   // free once the reduction is done
    {
      unsigned dsm;
      asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
      const size_t per = tri_ws_bytes(n);          // this CTA's other sample slots hold S x
      if (dsm > per) {
        ap.ys = reinterpret_cast<float2*>(smem + per);
        ap.ys_cap = (int)((dsm - per) / sizeof(float2));
      }
    }
    // mixed path with a CTA of three or more warps: float-float steps 2-5
    res = tri_smallest<double, true>(W, G, n, far, 1, gap, ap, tk, false, nullptr,
                                     a.mixed && blockDim.x >= 96);
    if (warp != 0) return;
  } else {
    SylvesterApply<false> ap;
    ap.P = sample_polys<double, double>(a.pz[ps], a.len[ps], f, a.C, a.ns, s);
    ap.C = a.C;
    ap.t1 = a.t1;
    ap.t2 = a.t2;
    ap.L = a.len[ps][0] + a.t2 - 1;
    ap.y = a.resid + o * a.C * (int64_t)a.Lmax;
    ap.F[0] = ap.F[1] = nullptr;
    if (a.mixed) {   // the mixed path keeps complex samples as float-float pairs only
      for (int k = 0; k < 2; ++k) {
        ap.F[k] = a.pzf[ps][k] + ((int64_t)f * a.C * a.ns + s) * a.len[ps][k];
        ap.fstride[k] = (int64_t)a.len[ps][k] * a.ns;
      }
    }
    ap.real = false;
    // mixed path: single-precision T and Newton steps against G first
    res = tri_smallest<cd, false>(W, G, n, far, 1, gap, ap, tk, a.mixed != 0);
  }
#ifdef CBP_PHASE_TIMING
  if (tk && lane == 0)
    printf("tri pass=%d s=%d real=%d near=%d | reduce %lld bisect %lld invit %lld newton %lld "
           "(apply %lld) theta %lld\n", ps, s, (int)real, res.near_degenerate, tkv[1] - tkv[0],
           tkv[2] - tkv[1], tkv[3] - tkv[2], tkv[4] - tkv[3], tkv[6] ? tkv[6] - tkv[3] : 0,
           tkv[5] - tkv[4]);
#endif
  for (int i = lane; i < n; i += 32) a.X[o * n + i] = W.x[i];
#ifdef CBP_SCHED_TRACE
  if (lane == 0) {
    unsigned long long t_end;
    unsigned smid;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    printf("SCHED %d %d %d %d %u %llu %llu %d\n", (int)real, f, ps, s, smid, t_start, t_end,
           (int)res.near_degenerate);
  }
#endif
  if (lane == 0) {
    a.sdiag[o * 4 + 0] = res.lam_max;
    a.sdiag[o * 4 + 1] = res.lam_2;
    a.sdiag[o * 4 + 2] = res.theta;
    a.sdiag[o * 4 + 3] = res.near_degenerate;
  }
}

// ------------------------------------------------- scale fix and kernels ---
struct ScaleArgs {
  const cd* X;          // [n][2][ns][nn]
  const double* sdiag;  // [n][2][ns][4]
  const int* bad;       // [n]
  const int* err;       // set when a copy of an earlier kernel did not complete in time
  cd* ab;               // [n][4][M][M]  A_1, A_2, B_1, B_2
  double* kd;           // [n][t1*t1 + t2*t2]
  void* k1_out;
  void* k2_out;
  const uint64_t* k1_tab;   // optional per-pair kernel addresses
  const uint64_t* k2_tab;
  int out_f64;
  cbp_diag* diag;       // [n]
  const int* accepted;  // learned path: proposal passed the gate (kernels already in kd)
  const double* rho;    // learned path: consistency residual of the proposal
  int M, ns, t1, t2, nn, mixed, Ph, Pw;
  int mode;             // kScaleLS, kScaleK1, kScaleSupport
  int ffx;              // mixed path with room for the float-float stage (scale_ff_offset)
};

// Scale fixes: both kernels' two-order least squares; kernel 1's equations
// only (the paper's k1-only pipeline); the single-pass support constraint.
constexpr int kScaleLS = 0, kScaleK1 = 1, kScaleSupport = 2;

// w^k (sign -1) or w^-k (sign +1), w = exp(-2 pi i / M), from a table of w^j, j < M.
__device__ __forceinline__ cd root(const cd* wt, int k, int M, double sign) {
  const cd w = wt[k % M];
  return sign < 0 ? w : conj(w);
}

// Cofactor of kernel kk (0, 1) at sample s of pass ps, conjugate-expanded.
__device__ __forceinline__ cd cofactor(const ScaleArgs& a, int f, int ps, int s, int idx) {
  const int M = a.M;
  const bool cj = s >= a.ns;
  const int ss = cj ? M - s : s;
  cd v = a.X[(((int64_t)f * 2 + ps) * a.ns + ss) * a.nn + idx];
  return cj ? conj(v) : v;
}

// Exact S^H S theta for the scale system (rows: gamma_j A_k[i][j] - delta_i B_k[i][j]).
struct ScaleApply {
  const cd* ab;
  int M;
  int nk;               // kernels whose equations enter (2, or 1 for the k1-only fix)
  __device__ void operator()(const cd* th, cd* out) const {
    const int MM = M * M;
    for (int u = threadIdx.x; u < 2 * M; u += blockDim.x) {
      cd acc = mk(0.0, 0.0);
      for (int k = 0; k < nk; ++k) {
        const cd* A = ab + k * MM;
        const cd* B = ab + (2 + k) * MM;
        for (int t = 0; t < M; ++t) {
          int i = u < M ? t : u - M;
          int j = u < M ? u : t;
          cd res = th[j] * A[i * M + j] - th[M + i] * B[i * M + j];
          if (u < M) cfmac(acc, A[i * M + j], res);
          else {
            cd v = mk(0.0, 0.0);
            cfmac(v, B[i * M + j], res);
            acc = acc - v;
          }
        }
      }
      out[u] = acc;
    }
    __syncthreads();
  }
};

// Exact operator of the support-constrained system (rows r_j = A_k[i][j] w^(-j q),
// k = 1, 2, every i, t_k <= q < M): out = S^H (S theta), S theta staged in s.
struct SupportApply {
  const cd* ab;
  const cd* wt;
  cd* s;                // [2][M][M] scratch (k, i, q)
  int M, t1, t2;
  __device__ void operator()(const cd* th, cd* out) const {
    const int MM = M * M;
    for (int e = threadIdx.x; e < 2 * MM; e += blockDim.x) {
      const int k = e / MM, i = (e % MM) / M, q = e % M;
      cd acc = mk(0.0, 0.0);
      if (q >= (k ? t2 : t1))
        for (int j = 0; j < M; ++j) cfma(acc, ab[k * MM + i * M + j] * root(wt, j * q, M, 1.0), th[j]);
      s[e] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      cd acc = mk(0.0, 0.0);
      for (int k = 0; k < 2; ++k)
        for (int i = 0; i < M; ++i)
          for (int q = k ? t2 : t1; q < M; ++q)
            cfmac(acc, ab[k * MM + i * M + j] * root(wt, j * q, M, 1.0), s[k * MM + i * M + q]);
      out[j] = acc;
    }
    __syncthreads();
  }
};

// Shared memory of k_scale_solve: the normal matrix (2M x 2M complex), block
// reduction scratch (32 doubles), X and T (3 M^2 complex), then the
// tridiagonal solver's work area.
__host__ __device__ inline size_t scale_tri_offset(int M) {
  return (sizeof(cd) * 4 * M * M + 32 * sizeof(double) + sizeof(cd) * 3 * M * M + 127) &
         ~size_t(127);
}
// then the mixed path's float-float cofactors [2][M][nn] and lifted spectra [4][M][M]
__host__ __device__ inline size_t scale_ff_offset(int M, int nn) {
  return (scale_tri_offset(M) + tri_ws_bytes(2 * M) + 127) & ~size_t(127);
}
__host__ __device__ inline size_t scale_ff_bytes(int M, int nn) {
  return sizeof(cfx) * (2 * (size_t)M * nn + 4 * (size_t)M * M);
}

__global__ void __launch_bounds__(kSolveThreads) k_scale_solve(ScaleArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int f = blockIdx.x;
  if (a.accepted && a.accepted[f]) {
    // learned path, proposal accepted: its kernels (in kd) are the result
    const int per = a.t1 * a.t1 + a.t2 * a.t2;
    const double* kd = a.kd + (int64_t)f * per;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int k = e >= a.t1 * a.t1, t = k ? a.t2 : a.t1, ek = k ? e - a.t1 * a.t1 : e;
      void* out = k ? a.k2_out : a.k1_out;
      int64_t oi = (int64_t)f * t * t + ek;
      const uint64_t* tab = k ? a.k2_tab : a.k1_tab;
      if (tab) {
        out = (void*)tab[f];
        oi = ek;
      }
      if (out) {
        if (a.out_f64) ((double*)out)[oi] = kd[e];
        else ((float*)out)[oi] = (float)kd[e];
      }
    }
    if (threadIdx.x == 0) {
      cbp_diag d = {};
      d.rho = a.rho[f];
      d.used_fallback = 0;
      d.pad_h = a.Ph;
      d.pad_w = a.Pw;
      d.status = *a.err ? CBP_ERR_TIMEOUT : a.bad[f] ? CBP_ERR_INVALID_ARG : CBP_OK;
      a.diag[f] = d;
    }
    return;
  }
  const int M = a.M, MM = M * M, t1 = a.t1, t2 = a.t2;
  const int mode = a.mode;
  const int n = mode == kScaleSupport ? M : 2 * M;   // unknowns: gamma (support) or (gamma, delta)
  const int nk = mode == kScaleK1 ? 1 : 2;            // kernels estimated
#ifdef CBP_PHASE_TIMING
  long long ph[8] = {0, 0, 0, 0, 0, 0, 0, 0}, tkv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long* tk = f < 2 ? tkv : nullptr;
#else
  long long* tk = nullptr;
#endif
  CBP_TICK(ph, 0);
  cd* Gs = (cd*)smem;                   // [n][n] normal matrix
  double* red = (double*)(Gs + n * n);   // block reductions
  char* p = (char*)(red + 32);
  cd* X = (cd*)p;                 // [2][M][M] kernel spectra, then full inverse DFTs
  cd* T = X + 2 * MM;             // [M][M] temporary
  __shared__ cd wt[kMaxM];
  __shared__ cfx wtx[kMaxM];
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)M, &sn, &cs);
    wt[k] = mk(cs, sn);
    wtx[k] = cfx_of(wt[k]);
  }
  __syncthreads();
  cd* ab = a.ab + (int64_t)f * 4 * MM;
  // Mixed path (two-order and k1-only fixes): the lift, the normal matrix and
  // the inverse DFT in float-float arithmetic (~1e-14) on the single-precision
  // units, the cofactors and lifted spectra staged in shared memory.
  const bool ffx = a.ffx && mode != kScaleSupport;
  cfx* cof = (cfx*)(smem + scale_ff_offset(M, a.nn));   // [2][M][nn] cofactors, conjugates expanded
  cfx* abx = cof + 2 * M * a.nn;                         // [4][M][M] A_1, A_2, B_1, B_2
  if (ffx) {
    for (int idx = threadIdx.x; idx < 2 * M * a.nn; idx += blockDim.x) {
      const int ps = idx / (M * a.nn), sm = (idx / a.nn) % M, e = idx % a.nn;
      cof[idx] = cfx_of(cofactor(a, f, ps, sm, e));
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 4 * MM; idx += blockDim.x) {
      const int which = idx / MM, i = (idx % MM) / M, j = idx % M;
      const int kk = which & 1, isB = which >> 1;
      const int t = kk ? t2 : t1, lo = kk ? t1 : 0;
      const cfx* u = cof + ((isB ? M : 0) + (isB ? i : j)) * a.nn + lo;
      const int mult = isB ? j : i;
      cfx_acc acc;
      for (int q = 0; q < t; ++q) acc.mac(u[q], wtx[(mult * q) % M]);
      const cfx v = acc.value();
      abx[idx] = v;
      ab[idx] = cfx_val(v);
    }
  }
  // lift: A_k[i][j] = sum_p u^{Z2}_{k,j}[p] w^{ip};  B_k[i][j] = sum_q u^{Z1}_{k,i}[q] w^{jq}
  for (int idx = threadIdx.x; !ffx && idx < 4 * MM; idx += blockDim.x) {
    const int which = idx / MM, i = (idx % MM) / M, j = idx % M;
    const int kk = which & 1, isB = which >> 1;
    const int t = kk ? t2 : t1, lo = kk ? t1 : 0;
    cd acc = mk(0.0, 0.0);
    for (int q = 0; q < t; ++q) {
      if (!isB) cfma(acc, cofactor(a, f, 0, j, lo + q), root(wt, i * q, M, -1.0));
      else cfma(acc, cofactor(a, f, 1, i, lo + q), root(wt, j * q, M, -1.0));
    }
    ab[idx] = acc;
  }
  __syncthreads();
  CBP_TICK(ph, 1);
  // normal matrix of the scale system
  if (ffx) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx % n;
      cfx_acc g;
      if (r < M && c < M) {
        if (r == c)
          for (int k = 0; k < nk; ++k)
            for (int i = 0; i < M; ++i) g.macc(abx[k * MM + i * M + r], abx[k * MM + i * M + r]);
      } else if (r >= M && c >= M) {
        if (r == c)
          for (int k = 0; k < nk; ++k)
            for (int j = 0; j < M; ++j)
              g.macc(abx[(2 + k) * MM + (r - M) * M + j], abx[(2 + k) * MM + (r - M) * M + j]);
      } else if (r < M) {   // (gamma_j, delta_i) = -sum_k conj(A_k[i][j]) B_k[i][j]
        const int j = r, i = c - M;
        for (int k = 0; k < nk; ++k) {
          const cfx av = abx[k * MM + i * M + j];
          g.macc({fx_neg(av.re), fx_neg(av.im)}, abx[(2 + k) * MM + i * M + j]);
        }
      } else {
        const int j = c, i = r - M;
        for (int k = 0; k < nk; ++k) {
          const cfx bv = abx[(2 + k) * MM + i * M + j];
          g.macc({fx_neg(bv.re), fx_neg(bv.im)}, abx[k * MM + i * M + j]);
        }
      }
      Gs[idx] = cfx_val(g.value());
    }
  }
  for (int idx = threadIdx.x; !ffx && idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx % n;
    cd g = mk(0.0, 0.0);
    if (mode == kScaleSupport) {
      // sum over rows (k, i, q >= t_k) of conj(A_k[i][r] w^-rq) A_k[i][c] w^-cq
      for (int k = 0; k < 2; ++k) {
        cd e = mk(0.0, 0.0);                   // sum_q w^((r - c) q), q = t_k .. M-1
        for (int q = k ? t2 : t1; q < M; ++q) e = e + root(wt, ((r - c + M) % M) * q, M, -1.0);
        cd h = mk(0.0, 0.0);
        for (int i = 0; i < M; ++i) cfmac(h, ab[k * MM + i * M + r], ab[k * MM + i * M + c]);
        g = g + h * e;
      }
    } else if (r < M && c < M) {
      if (r == c)
        for (int k = 0; k < nk; ++k)
          for (int i = 0; i < M; ++i) g.re += abs2(ab[k * MM + i * M + r]);
    } else if (r >= M && c >= M) {
      if (r == c)
        for (int k = 0; k < nk; ++k)
          for (int j = 0; j < M; ++j) g.re += abs2(ab[(2 + k) * MM + (r - M) * M + j]);
    } else if (r < M) {   // (gamma_j, delta_i) = -sum_k conj(A_k[i][j]) B_k[i][j]
      const int j = r, i = c - M;
      for (int k = 0; k < nk; ++k) {
        cd v = cmulc(ab[k * MM + i * M + j], ab[(2 + k) * MM + i * M + j]);
        g = g - v;
      }
    } else {
      const int j = c, i = r - M;
      for (int k = 0; k < nk; ++k) {
        cd v = cmulc(ab[(2 + k) * MM + i * M + j], ab[k * MM + i * M + j]);
        g = g - v;
      }
    }
    Gs[idx] = g;
  }
  __syncthreads();
  CBP_TICK(ph, 2);
  // Null vector of the scale system by the warp-level tridiagonal solver, one
  // refinement step against the exact operator (FP64 path); the mixed path
  // takes its single-precision T with Newton steps against the double G.
  const TriWs W = carve_tri(smem + scale_tri_offset(M), n);
  cfx* Gx = nullptr;   // float-float copy of the normal matrix (the cofactors' space is free)
  if (ffx) {
    Gx = cof;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Gx[idx] = cfx_of(Gs[idx]);
    __syncthreads();
  }
  TriResult res;
  if (mode == kScaleSupport) {
    SupportApply ap{ab, wt, X, M, t1, t2};      // X is free until the combination below
    res = tri_smallest<cd, true>(W, Gs, n, 1, 1, 1e300, ap, tk, a.mixed != 0);
  } else {
    ScaleApply ap{ab, M, nk};
    res = tri_smallest<cd, true>(W, Gs, n, 1, 1, 1e300, ap, tk, a.mixed != 0, Gx);
  }
  __syncthreads();
  CBP_TICK(ph, 3);
  const cd* xs = W.x;
  // X_k[i][j] = (gamma_j A_k[i][j] + delta_i B_k[i][j]) / 2, or gamma_j A_k[i][j]
  // (support); the k1-only fix leaves kernel 2's spectrum zero
  for (int idx = threadIdx.x; idx < 2 * MM; idx += blockDim.x) {
    const int k = idx / MM, i = (idx % MM) / M, j = idx % M;
    if (k >= nk) X[idx] = mk(0.0, 0.0);
    else if (mode == kScaleSupport) X[idx] = xs[j] * ab[k * MM + i * M + j];
    else X[idx] = 0.5 * (xs[j] * ab[k * MM + i * M + j] + xs[M + i] * ab[(2 + k) * MM + i * M + j]);
  }
  __syncthreads();
  __shared__ cd x00[2];
  if (threadIdx.x < 2) x00[threadIdx.x] = X[threadIdx.x * MM];
  __syncthreads();
  CBP_TICK(ph, 4);
  // inverse DFT, separable: T[i][q] = sum_j X[i][j] w^{-jq};  K[p][q] = sum_i w^{-ip} T[i][q] / M^2
  for (int k = 0; k < 2; ++k) {
    if (k >= nk) {
      // k1-only: no kernel 2 (its internal copy zeroed, the caller's buffer untouched)
      double* kd2 = a.kd + (int64_t)f * (t1 * t1 + t2 * t2) + t1 * t1;
      for (int e = threadIdx.x; e < t2 * t2; e += blockDim.x) kd2[e] = 0.0;
      continue;
    }
    cd* Xk = X + k * MM;
    const cd inv00 = [&] {
      cd z = x00[k];
      double d = abs2(z);
      return d > 0 ? mk(z.re / d, -z.im / d) : mk(0.0, 0.0);
    }();
    cfx* Yx = (cfx*)Xk;   // float-float: Xk inv00 in place, then the stages on Tx
    cfx* Tx = (cfx*)T;
    if (ffx) {
      const cfx inv = cfx_of(inv00);
      for (int idx = threadIdx.x; idx < MM; idx += blockDim.x) Yx[idx] = cfx_mul(cfx_of(Xk[idx]), inv);
      __syncthreads();
      for (int idx = threadIdx.x; idx < MM; idx += blockDim.x) {
        const int i = idx / M, q = idx % M;
        cfx_acc acc;
        for (int j = 0; j < M; ++j) {
          const cfx w = wtx[(j * q) % M];
          acc.mac(Yx[i * M + j], {w.re, fx_neg(w.im)});
        }
        Tx[idx] = acc.value();
      }
    }
    for (int idx = threadIdx.x; !ffx && idx < MM; idx += blockDim.x) {
      const int i = idx / M, q = idx % M;
      cd acc = mk(0.0, 0.0);
      for (int j = 0; j < M; ++j) cfma(acc, Xk[i * M + j] * inv00, root(wt, j * q, M, 1.0));
      T[idx] = acc;
    }
    __syncthreads();
    const int t = k ? t2 : t1;
    double* kd = a.kd + (int64_t)f * (t1 * t1 + t2 * t2) + (k ? t1 * t1 : 0);
    double l_im = 0, l_re = 0, l_out = 0;
    for (int idx = threadIdx.x; idx < MM; idx += blockDim.x) {
      const int pp = idx / M, q = idx % M;
      cd acc = mk(0.0, 0.0);
      if (ffx) {
        cfx_acc ax;
        for (int i = 0; i < M; ++i) {
          const cfx w = wtx[(i * pp) % M];
          ax.mac({w.re, fx_neg(w.im)}, Tx[i * M + q]);
        }
        acc = cfx_val(ax.value());
      } else {
        for (int i = 0; i < M; ++i) cfma(acc, root(wt, i * pp, M, 1.0), T[i * M + q]);
      }
      acc = (1.0 / (double)MM) * acc;
      l_re += acc.re * acc.re;
      l_im += acc.im * acc.im;
      if (pp >= t || q >= t) l_out += abs2(acc);
      if (pp < t && q < t && CBP_CHECK(pp < a.M && q < a.M, 3)) {
        kd[pp * t + q] = acc.re;
        void* out = k ? a.k2_out : a.k1_out;
        int64_t oi = (int64_t)f * t * t + pp * t + q;
        const uint64_t* tab = k ? a.k2_tab : a.k1_tab;
        if (tab) {
          out = (void*)tab[f];
          oi = pp * t + q;
        }
        if (out) {
          if (a.out_f64) ((double*)out)[oi] = acc.re;
          else ((float*)out)[oi] = (float)acc.re;
        }
      }
    }
    l_re = block_sum(l_re, red);
    l_im = block_sum(l_im, red);
    l_out = block_sum(l_out, red);
    if (threadIdx.x == 0) {
      double ir = l_re > 0 ? sqrt(l_im / l_re) : 0.0;
      double sr = (l_re + l_im) > 0 ? l_out / (l_re + l_im) : 0.0;
      if (k == 0) {
        a.diag[f].imag_ratio = ir;
        a.diag[f].support_ratio = sr;
      } else {
        a.diag[f].imag_ratio = fmax(a.diag[f].imag_ratio, ir);
        a.diag[f].support_ratio = fmax(a.diag[f].support_ratio, sr);
      }
    }
    __syncthreads();
  }
  CBP_TICK(ph, 5);
#ifdef CBP_PHASE_TIMING
  if (tk && threadIdx.x == 0)
    printf("scale f=%d | lift %lld normal %lld tri %lld (reduce %lld bisect %lld invit %lld newton %lld "
           "theta %lld) combine %lld idft %lld\n", f, ph[1] - ph[0], ph[2] - ph[1], ph[3] - ph[2],
           tkv[1] - tkv[0], tkv[2] - tkv[1], tkv[3] - tkv[2], tkv[4] - tkv[3], tkv[5] - tkv[4],
           ph[4] - ph[3], ph[5] - ph[4]);
#endif
  // aggregate diagnostics
  if (threadIdx.x == 0) {
    double kappa = 0, gap = 1e300, smin = 0;
    int flagged = 0, hard = 0;
    for (int i = 0; i < 2 * a.ns; ++i) {
      const double* d = a.sdiag + ((int64_t)f * 2 * a.ns + i) * 4;
      const double lmax = d[0] > 0 ? d[0] : 1e-300;
      const double g = sqrt(fmax(d[1], 0.0) / lmax);
      gap = fmin(gap, g);
      kappa = fmax(kappa, g > 0 ? 1.0 / g : 1e300);
      smin = fmax(smin, sqrt(fmax(d[2], 0.0) / lmax));
      if (g < 1e-8) ++flagged;
      hard += (int)d[3];
    }
    cbp_diag& dg = a.diag[f];
    dg.kappa_max = kappa;
    dg.gap_min = gap;
    dg.sigma_min_max = smin;
    dg.scale_resid = sqrt(fmax(res.theta, 0.0) / fmax(res.lam_max, 1e-300));
    dg.rho = a.rho ? a.rho[f] : 0.0;
    dg.flagged_samples = flagged;
    dg.used_fallback = a.accepted ? 1 : 0;
    dg.pad_h = a.Ph;
    dg.pad_w = a.Pw;
    dg.hard_samples = hard;
    int st = CBP_OK;
    if (*a.err) st = CBP_ERR_TIMEOUT;
    else if (a.bad[f]) st = CBP_ERR_INVALID_ARG;
    else if (!(x00[0].re != 0.0 || x00[0].im != 0.0) ||
             (nk > 1 && !(x00[1].re != 0.0 || x00[1].im != 0.0)))
      st = CBP_ERR_NOT_COPRIME;
    else if (gap < 1e-13) st = CBP_ERR_NOT_COPRIME;
    else if (flagged) st = CBP_WARN_ILL_CONDITIONED;
    dg.status = st;
  }
}

__global__ void k_kernels_in(const void* k1, const void* k2, int in_f64, int n, int t1, int t2,
                             double* kd, cbp_diag* diag, int Ph, int Pw, const int* bad,
                             const uint64_t* k1_tab, const uint64_t* k2_tab) {
  const int per = t1 * t1 + t2 * t2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * per;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(i / per), e = (int)(i % per);
    // kernel k of pair f: from the table if given, else the contiguous batch
    const bool second = e >= t1 * t1;
    const int tk = second ? t2 : t1, ek = second ? e - t1 * t1 : e;
    const uint64_t* tab = second ? k2_tab : k1_tab;
    const void* base = tab ? (const void*)tab[f] : (second ? k2 : k1);
    const int64_t o = tab ? ek : (int64_t)f * tk * tk + ek;
    const double v = in_f64 ? ((const double*)base)[o] : (double)((const float*)base)[o];
    kd[i] = v;
    if (e == 0) {
      cbp_diag d = {};
      d.pad_h = Ph;
      d.pad_w = Pw;
      d.status = bad && bad[f] ? CBP_ERR_INVALID_ARG : CBP_OK;
      diag[f] = d;
    }
  }
}

// ------------------------------------------------- kernel-size estimation ---
// The kernel degree (Section 4: read from the singularity of the cofactor
// system; Section 5: a scan of candidate sizes with a fallback to the
// largest).  Under full convolution the blurred sizes fix d = t1 - t2; for
// candidate t1' (t2' = t1' - d) the Sylvester system of the z = 1 samples
// (row sums, column sums) has a null vector exactly when t1' >= t1.  One CTA
// per (candidate, order, pair) forms the real normal matrix from the
// correlations and takes its extreme eigenvalues with the tridiagonal solver
// (no refinement steps): ratio = sqrt(theta / lambda_max), theta the
// Rayleigh quotient of the smallest eigenvector.

// z = 1 samples of a frame batch: row sums [n][C][h] and column sums
// [n][C][w] (imaginary parts zero), accumulated in double.
__global__ void k_plane_sums(FrameDesc fr, cd* rows, cd* cols) {
  const int fc = blockIdx.y, f = fc / fr.c, ch = fc % fr.c;
  const char* base = (const char*)frame_base(fr, f) + (int64_t)ch * fr.cs * (fr.f64 ? 8 : 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (blockIdx.z == 0) {
    for (int r = blockIdx.x * nw + warp; r < fr.h; r += gridDim.x * nw) {
      double acc = 0.0;
      for (int c = lane; c < fr.w; c += 32) acc += ld_frame<double>(base, (int64_t)r * fr.rs + c, fr.f64);
      acc = warp_sum(acc);
      if (lane == 0) rows[(int64_t)fc * fr.h + r] = mk(acc, 0.0);
    }
  } else {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < fr.w; c += gridDim.x * blockDim.x) {
      double acc = 0.0;
      for (int r = 0; r < fr.h; ++r) acc += ld_frame<double>(base, (int64_t)r * fr.rs + c, fr.f64);
      cols[(int64_t)fc * fr.w + c] = mk(acc, 0.0);
    }
  }
}

struct SizeScanArgs {
  const cd* pz[2][2];   // [order][frame]: z = 1 samples [n][C][len]
  int len[2][2];
  int C, t_min, d, ncand;
  double* ratio;        // [n][2][ncand]; -1 for an invalid candidate
};

// The refinement steps are off in the scan: an operator that is never applied.
struct NoApply {
  __device__ void operator()(const cd*, cd*) const {}
};

__global__ void __launch_bounds__(kSolveThreads) k_size_scan(SizeScanArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int cand = blockIdx.x, ps = blockIdx.y, f = blockIdx.z;
  const int t1 = a.t_min + cand, t2 = t1 - a.d, n = t1 + t2;
  double* out = a.ratio + ((int64_t)f * 2 + ps) * a.ncand + cand;
  if (t1 < 1 || t2 < 1 || n > kMaxN || n < 2) {
    if (threadIdx.x == 0) *out = -1.0;
    return;
  }
  cd* G = (cd*)smem;                                    // [n][n]
  cd* rho = G + kMaxN * kMaxN;                          // [2 n - 1]
  const TriWs W = carve_tri(smem + sizeof(cd) * (kMaxN * kMaxN + 2 * kMaxN), n);
  const SamplePolys<double, double> P = sample_polys<double, double>(a.pz[ps], a.len[ps], f, a.C, 1, 0);
  correlations_real(P, a.C, t1, t2, rho);
  gram_from_rho(rho, t1, t2, G);
  const TriResult res = tri_smallest<double, true>(W, G, n, 0, 0, 1e300, NoApply{});
  // the Rayleigh quotient of the converged vector (the multisection bracket
  // is only narrowed as far as the eigenvector needs)
  if (threadIdx.x == 0) *out = res.lam_max > 0.0 ? sqrt(fmax(res.theta, 0.0) / res.lam_max) : 0.0;
}

// Per pair: the smallest candidate whose ratio (the larger of the two
// orders') is at most tol, else the largest valid candidate.
__global__ void k_size_pick(const double* ratio, int n, int ncand, int t_min, int d, double tol,
                            int* t_out /* [n][3]: t1, t2, found */, double* rmax /* [n][ncand] */) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  int best = -1, last = -1;
  for (int c = 0; c < ncand; ++c) {
    const double r0 = ratio[((int64_t)f * 2 + 0) * ncand + c];
    const double r1 = ratio[((int64_t)f * 2 + 1) * ncand + c];
    const bool valid = r0 >= 0.0 && r1 >= 0.0;
    rmax[(int64_t)f * ncand + c] = valid ? fmax(r0, r1) : -1.0;
    if (!valid) continue;
    last = c;
    if (best < 0 && fmax(r0, r1) <= tol) best = c;
  }
  const int c = best >= 0 ? best : last;
  t_out[3 * f + 0] = c >= 0 ? t_min + c : 0;
  t_out[3 * f + 1] = c >= 0 ? t_min + c - d : 0;
  t_out[3 * f + 2] = best >= 0 ? 1 : 0;
}

// ------------------------------------------- coprimality of kernel pairs ---
// The camera side's test (Section 3: the pair must be coprime as bivariate
// polynomials): at every solved sample w^j (j <= M/2; sample M - j is the
// conjugate) of both evaluation orders, the univariate polynomials
// a = K1(., w^j), b = K2(., w^j) share no root -- sigma_min / sigma_max of
// their square Sylvester matrix (the cofactor system at t1 - 1, t2 - 1)
// above tol, from its normal matrix's extreme eigenvalues -- and one of them
// keeps full degree (|leading coefficient| > 1e-12 of its norm).
struct CoprimeArgs {
  const double* ka;     // [n][ta ta]
  const double* kb;     // [n][tb tb]
  int ta, tb, M, ns;
  const int* active;    // [n] pairs under test
  double tol;
  int* pass;            // [n][2][ns]
};

__global__ void __launch_bounds__(kSolveThreads) k_coprime_test(CoprimeArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int j = blockIdx.x, order = blockIdx.y, f = blockIdx.z;
  if (!a.active[f]) return;
  const int ta = a.ta, tb = a.tb, n = ta + tb - 2;
  cd* pa = (cd*)smem;                                  // [ta]
  cd* pb = pa + kMaxN;                                 // [tb]
  cd* G = pb + kMaxN;                                  // [n][n]
  cd* rho = G + kMaxN * kMaxN;                         // [2 n - 1]
  __shared__ int full;
  const double* K1 = a.ka + (int64_t)f * ta * ta;
  const double* K2 = a.kb + (int64_t)f * tb * tb;
  // a[p] = sum_q K1[p][q] w^(j q) (order 0) or a[q] = sum_p K1[p][q] w^(j p)
  for (int e = threadIdx.x; e < ta + tb; e += blockDim.x) {
    const bool second = e >= ta;
    const int t = second ? tb : ta, i = second ? e - ta : e;
    const double* K = second ? K2 : K1;
    cd acc = mk(0.0, 0.0);
    for (int k = 0; k < t; ++k) {
      double sn, cs;
      sincospi(-2.0 * (double)((j * k) % a.M) / (double)a.M, &sn, &cs);
      const double v = order == 0 ? K[i * t + k] : K[k * t + i];
      acc = acc + v * mk(cs, sn);
    }
    (second ? pb : pa)[i] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double na = 0.0, nb = 0.0;
    for (int i = 0; i < ta; ++i) na += abs2(pa[i]);
    for (int i = 0; i < tb; ++i) nb += abs2(pb[i]);
    full = (abs2(pa[ta - 1]) > 1e-24 * na) || (abs2(pb[tb - 1]) > 1e-24 * nb);
  }
  __syncthreads();
  double ratio = 1.0;
  if (ta > 1 && tb > 1) {
    SamplePolys<double, double> P;
    P.c[0] = pa;
    P.c[1] = pb;
    P.cstride[0] = P.cstride[1] = 0;
    P.len[0] = ta;
    P.len[1] = tb;
    correlations(P, 1, ta - 1, tb - 1, rho);
    gram_from_rho(rho, ta - 1, tb - 1, G);
    const TriWs W = carve_tri(smem + sizeof(cd) * (2 * kMaxN + kMaxN * kMaxN + 2 * kMaxN), n);
    const TriResult res = tri_smallest<cd, true>(W, G, n, 0, 0, 1e300, NoApply{});
    ratio = res.lam_max > 0.0 ? sqrt(fmax(res.theta, 0.0) / res.lam_max) : 0.0;
  }
  if (threadIdx.x == 0) a.pass[((int64_t)f * 2 + order) * a.ns + j] = (full && ratio > a.tol) ? 1 : 0;
}

// Per pair under test: accepted when every sample passed; else the next
// attempt, or -1 once max_attempts draws have failed.  *any: some pair is
// still under test.
__global__ void k_coprime_pick(int n, int ns, const int* pass, int* active, int* attempt,
                               int max_attempts, int* any) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n || !active[f]) return;
  bool ok = true;
  for (int i = 0; i < 2 * ns; ++i) ok = ok && pass[(int64_t)f * 2 * ns + i];
  if (ok) {
    active[f] = 0;
  } else if (attempt[f] + 1 < max_attempts) {
    attempt[f] += 1;
    atomicOr(any, 1);
  } else {
    active[f] = 0;
    attempt[f] = -1;
  }
}

// The solver's guarded reciprocal and reciprocal square root, elementwise.
__global__ void k_check_recip(const double* x, int64_t n, double* r, double* q) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    r[i] = rcp_safe(x[i]);
    q[i] = x[i] > 0.0 ? rsqrt_safe(x[i]) : 0.0;
  }
}

}  // namespace

size_t sample_solve_smem(int nn) { return tri_ws_bytes(nn); }
size_t scale_solve_smem(int M, int nn) { return scale_tri_offset(M) + tri_ws_bytes(2 * M); }

void launch_sample_solve(const Plan& p, char* ws, cudaStream_t st) {
  SampleArgs a;
  for (int k = 0; k < 2; ++k) {
    a.pz[0][k] = (const cd*)(ws + p.off_pz2[k]);
    a.pz[1][k] = (const cd*)(ws + p.off_pz1[k]);
    a.pzf[0][k] = p.mixed ? (const cdf*)(ws + p.off_pz2f[k]) : nullptr;
    a.pzf[1][k] = p.mixed ? (const cdf*)(ws + p.off_pz1f[k]) : nullptr;
  }
  a.len[0][0] = p.H1;
  a.len[0][1] = p.H2;
  a.len[1][0] = p.W1;
  a.len[1][1] = p.W2;
  a.X = (cd*)(ws + p.off_x);
  a.sdiag = (double*)(ws + p.off_sdiag);
  a.resid = (cd*)(ws + p.off_resid);
  a.Lmax = p.Lmax;
  a.C = p.C;
  a.ns = p.ns;
  a.t1 = p.t1;
  a.t2 = p.t2;
  a.nn = p.nn;
  a.M = p.M;
  a.mixed = p.mixed;
  a.accepted = p.learned ? (const int*)(ws + p.off_acc) : nullptr;
  a.G = (cd*)(ws + p.off_gall);
  dim3 grid(p.n, 2, p.ns);
  k_sample_gram<<<grid, kSolveThreads, 0, st>>>(a);
  // warps (samples) per CTA: up to CBP_SOLVE_WPC within ~110 KB of shared memory
  const int nrs = (p.M % 2 == 0) ? 2 : 1, ncs = p.ns - nrs;
  const int nreal = p.n * 2 * nrs, ncomplex = p.n * 2 * ncs;
  const size_t per = tri_ws_bytes(p.nn);
  const int wpc = (int)std::max<size_t>(1, std::min<size_t>(CBP_SOLVE_WPC, (110u << 10) / per));
  const size_t sm = per * wpc;
  a.nfr = p.n;
  cudaFuncSetAttribute(k_sample_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_sample_solve<<<nreal + (ncomplex + wpc - 1) / wpc, 32 * wpc, sm, st>>>(a, nreal);
}

void launch_scale_solve(const Plan& p, char* ws, void* k1_out, void* k2_out, int out_f64,
                        cudaStream_t st, const uint64_t* k1_tab, const uint64_t* k2_tab) {
  ScaleArgs a;
  a.X = (const cd*)(ws + p.off_x);
  a.sdiag = (const double*)(ws + p.off_sdiag);
  a.bad = (const int*)(ws + p.off_bad);
  a.err = (const int*)(ws + p.off_err);
  a.ab = (cd*)(ws + p.off_resid);  // reuses the residual scratch (sized for both)
  a.kd = (double*)(ws + p.off_kd);
  a.k1_out = k1_out;
  a.k2_out = k2_out;
  a.k1_tab = k1_tab;
  a.k2_tab = k2_tab;
  a.out_f64 = out_f64;
  a.diag = (cbp_diag*)(ws + p.off_diag);
  a.M = p.M;
  a.ns = p.ns;
  a.t1 = p.t1;
  a.t2 = p.t2;
  a.nn = p.nn;
  a.mixed = p.mixed;
  a.Ph = p.Ph;
  a.Pw = p.Pw;
  a.accepted = p.learned ? (const int*)(ws + p.off_acc) : nullptr;
  a.rho = p.learned ? (const double*)(ws + p.off_rho) : nullptr;
  a.mode = p.scale_mode;
  // the mixed path's float-float stage where its shared memory fits
  const size_t ff_end = scale_ff_offset(p.M, p.nn) + scale_ff_bytes(p.M, p.nn);
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  a.ffx = p.mixed && p.scale_mode != kScaleSupport && ff_end <= (size_t)smem_max;
  const size_t sm = a.ffx ? ff_end : scale_solve_smem(p.M, p.nn);
  cudaFuncSetAttribute(k_scale_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_scale_solve<<<p.n, kSolveThreads, sm, st>>>(a);
}

void launch_kernels_in(const Plan& p, char* ws, const void* k1, const void* k2, int in_f64,
                       cudaStream_t st, const uint64_t* k1_tab, const uint64_t* k2_tab) {
  const int64_t total = (int64_t)p.n * (p.t1 * p.t1 + p.t2 * p.t2);
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_kernels_in<<<blocks, 256, 0, st>>>(k1, k2, in_f64, p.n, p.t1, p.t2, (double*)(ws + p.off_kd),
                                       (cbp_diag*)(ws + p.off_diag), p.Ph, p.Pw,
                                       (const int*)(ws + p.off_bad), k1_tab, k2_tab);
}

size_t size_scan_smem() {
  return sizeof(cd) * (kMaxN * kMaxN + 2 * kMaxN) + tri_ws_bytes(kMaxN);
}

void launch_size_scan(const SizePlan& sp, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                      cudaStream_t st) {
  const FrameDesc* fr[2] = {&b1, &b2};
  for (int k = 0; k < 2; ++k) {
    dim3 g(std::max(1, std::min(64, (std::max(fr[k]->h, fr[k]->w) + 255) / 256)), sp.n * sp.C, 2);
    k_plane_sums<<<g, 256, 0, st>>>(*fr[k], (cd*)(ws + sp.off_rows[k]), (cd*)(ws + sp.off_cols[k]));
  }
  SizeScanArgs a;
  for (int k = 0; k < 2; ++k) {
    a.pz[0][k] = (const cd*)(ws + sp.off_rows[k]);
    a.pz[1][k] = (const cd*)(ws + sp.off_cols[k]);
  }
  a.len[0][0] = b1.h;
  a.len[0][1] = b2.h;
  a.len[1][0] = b1.w;
  a.len[1][1] = b2.w;
  a.C = sp.C;
  a.t_min = sp.t_min;
  a.d = sp.d;
  a.ncand = sp.ncand;
  a.ratio = (double*)(ws + sp.off_ratio);
  const size_t sm = size_scan_smem();
  cudaFuncSetAttribute(k_size_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_size_scan<<<dim3(sp.ncand, 2, sp.n), kSolveThreads, sm, st>>>(a);
  k_size_pick<<<(sp.n + 127) / 128, 128, 0, st>>>(a.ratio, sp.n, sp.ncand, sp.t_min, sp.d, sp.tol,
                                                 (int*)(ws + sp.off_t), (double*)(ws + sp.off_rmax));
}

size_t coprime_test_smem() {
  return sizeof(cd) * (2 * kMaxN + kMaxN * kMaxN + 2 * kMaxN) + tri_ws_bytes(kMaxN);
}

void launch_coprime_round(const double* ka, const double* kb, int n, int ta, int tb, int M,
                          double tol, int max_attempts, int* active, int* attempt, int* pass,
                          int* any, cudaStream_t st) {
  CoprimeArgs a;
  a.ka = ka;
  a.kb = kb;
  a.ta = ta;
  a.tb = tb;
  a.M = M;
  a.ns = M / 2 + 1;
  a.active = active;
  a.tol = tol;
  a.pass = pass;
  const size_t sm = coprime_test_smem();
  cudaFuncSetAttribute(k_coprime_test, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_coprime_test<<<dim3(a.ns, 2, n), kSolveThreads, sm, st>>>(a);
  k_coprime_pick<<<(n + 127) / 128, 128, 0, st>>>(n, a.ns, pass, active, attempt, max_attempts, any);
}

void launch_check_recip(const double* x, int64_t n, double* r, double* q, cudaStream_t st) {
  const int64_t b = (n + 255) / 256;
  k_check_recip<<<(int)std::min<int64_t>(std::max<int64_t>(b, 1), 4096), 256, 0, st>>>(x, n, r, q);
}

}  // namespace cbp
