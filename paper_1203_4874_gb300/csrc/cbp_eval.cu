// A1: evaluation of both blurred frames' bivariate z-polynomials at the M-th
// roots of unity, in both orders (Eq. 3; Section 5, "polynomial evaluation").
//
//   z2 = w^s  (rows kept):     P_Z2[s][r] = sum_c B[r][c] w^(s c)
//   z1 = w^s  (columns kept):  P_Z1[s][c] = sum_r B[r][c] w^(s r),   w = exp(-2 pi i / M)
//
// Because w^(s c) depends only on c mod M, each row (column) is first folded
// into M bins -- Fz2[m][r] = sum_{c = m mod M} B[r][c] -- and the M-point DFT
// of the bins gives every sample.  The folds run in the row pass
// (k_row_pass, cbp_fft.cu), which reads each frame row once, coalesced, and
// in a deblurring call also feeds the same rows to the deconvolution's row
// FFTs; this file turns the bins into samples.  Only samples s <= M/2 are
// produced (real input: sample M - s is the conjugate of sample s).  The
// paper's own kernel (Section 5, one thread block per row/column, one
// shared-memory reduction per sample) re-reads the frame once per sample; the
// fold makes the cost independent of M.
//
// Float32 frames are folded with an exact float TwoSum accumulation (hi + lo),
// so the bins -- and the samples -- carry ~1e-14 relative error on both paths.
// The FP64 path takes the M-point DFT in double precision.  The mixed path
// takes it in float-float arithmetic on the single-precision units (a GPU's
// double pipe is narrow) and keeps the samples as float-float pairs (its
// Gram is float-float too); double copies are written for the real samples
// (z = 1, z = -1), whose Gram and refinement run in double precision.
#include "cbp_common.cuh"
#include "cbp_internal.h"

namespace cbp {

CBP_CHECKS_TU(kChkEval)

namespace {

constexpr int kDftThreads = 128;

struct FoldDftArgs {
  const void* bins[4];     // [pass * 2 + frame]; pass 0: row bins, 1: column bins; [n C][M][len]
  cd* pz[4];               // [n C][ns][len] samples
  cdf* pzf[4];             // float-float copies (mixed path) or null
  int len[4];
  int M, ns;
  int pz_all;              // float-float kernel: double copies of every sample, not only the real ones
  const int* accepted;     // learned path: pairs whose proposal passed the gate (skipped), or null
  int C;
};

// 8-byte bin m of a position: (hi, lo) floats (F32) or a double.
template <bool F32>
__device__ __forceinline__ double bin_at(const void* b, int64_t i) {
  if (F32) {
    const float2 v = ((const float2*)b)[i];
    return (double)v.x + (double)v.y;
  }
  return ((const double*)b)[i];
}

// M-point DFT of each position's M real bins, samples s < ns, using the
// symmetry of the roots: with e_m = b_m + b_(M-m), o_m = b_m - b_(M-m),
//   P_s = b_0 + sum_{m=1..(M-1)/2} (e_m cos(2 pi s m / M) - i o_m sin(2 pi s m / M))
//         [+ (-1)^s b_(M/2) when M is even].
template <bool F32>
__global__ void __launch_bounds__(kDftThreads) k_fold_dft(FoldDftArgs a) {
  if (a.accepted && a.accepted[blockIdx.y / a.C]) return;   // the proposal stands (whole block)
  if (!CBP_CHECK(a.M <= kMaxM && a.ns <= a.M, 0)) return;    // the root tables' size (whole block)
  __shared__ double cs[kMaxM], sn[kMaxM];
  for (int k = threadIdx.x; k < a.M; k += blockDim.x) sincospi(2.0 * (double)k / (double)a.M, &sn[k], &cs[k]);
  __syncthreads();
  const int z = blockIdx.z, fc = blockIdx.y, M = a.M, len = a.len[z];
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= len) return;
  const int64_t b = (int64_t)fc * M * len + pos;
  const void* bb = a.bins[z];
  const int h = (M - 1) / 2;
  const double b0 = bin_at<F32>(bb, b);
  const double bh = (M % 2 == 0) ? bin_at<F32>(bb, b + (int64_t)(M / 2) * len) : 0.0;
  double ev[kMaxM / 2], od[kMaxM / 2];
#pragma unroll
  for (int m = 1; m <= kMaxM / 2; ++m) {
    if (m > h) break;
    const double u = bin_at<F32>(bb, b + (int64_t)m * len), v = bin_at<F32>(bb, b + (int64_t)(M - m) * len);
    ev[m - 1] = u + v;
    od[m - 1] = u - v;
  }
  cd* out = a.pz[z] + (int64_t)fc * a.ns * len + pos;
  cdf* outf = a.pzf[z] ? a.pzf[z] + (int64_t)fc * a.ns * len + pos : nullptr;
  for (int s = 0; s < a.ns; ++s) {
    double re = b0 + ((s & 1) ? -bh : bh), im = 0.0;
    int k = 0;
#pragma unroll
    for (int m = 1; m <= kMaxM / 2; ++m) {
      if (m > h) break;
      k += s;
      if (k >= M) k -= M;
      if (!CBP_CHECK(k >= 0 && k < M, 1)) k = 0;
      re = fma(ev[m - 1], cs[k], re);
      im = fma(-od[m - 1], sn[k], im);
    }
    const cd pv = mk(re, im);
    out[(int64_t)s * len] = pv;
    if (outf) outf[(int64_t)s * len] = to_cdf(pv);
  }
}

// Float-float arithmetic (hi + lo pairs of floats).
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {   // TwoSum of the high parts, low parts added
  const float s = a.hi + b.hi, z = s - a.hi;
  const float e = ((a.hi - (s - z)) + (b.hi - z)) + (a.lo + b.lo);
  const float hi = s + e;
  return {hi, e - (hi - s)};
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return {-a.hi, -a.lo}; }
// acc += a * c, the low part left unnormalised (renormalise once at the end):
// exact product of the high parts (FMA), cross terms, TwoSum into hi
__device__ __forceinline__ void f2_mac(F2& acc, F2 a, F2 c) {
  const float p = a.hi * c.hi;
  float e = fmaf(a.hi, c.hi, -p);
  e = fmaf(a.hi, c.lo, fmaf(a.lo, c.hi, e));
  const float t = acc.hi + p, z = t - acc.hi;
  acc.lo += ((acc.hi - (t - z)) + (p - z)) + e;
  acc.hi = t;
}
__device__ __forceinline__ F2 f2_norm(F2 a) {
  const float hi = a.hi + a.lo;
  return {hi, a.lo - (hi - a.hi)};
}

// The same DFT in float-float arithmetic from (hi, lo) bins of float32 frames:
// ~1e-14 of the terms' magnitudes, like the bins themselves.
__global__ void __launch_bounds__(kDftThreads, 4) k_fold_dft_ff(FoldDftArgs a) {
  if (a.accepted && a.accepted[blockIdx.y / a.C]) return;   // the proposal stands (whole block)
  if (!CBP_CHECK(a.M <= kMaxM && a.ns <= a.M, 0)) return;    // the root tables' size (whole block)
  __shared__ F2 cs[kMaxM], sn[kMaxM];
  for (int k = threadIdx.x; k < a.M; k += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)k / (double)a.M, &s, &c);
    const float ch = (float)c, sh = (float)s;
    cs[k] = {ch, (float)(c - (double)ch)};
    sn[k] = {sh, (float)(s - (double)sh)};
  }
  __syncthreads();
  const int z = blockIdx.z, fc = blockIdx.y, M = a.M, len = a.len[z];
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= len) return;
  const float2* bb = (const float2*)a.bins[z] + (int64_t)fc * M * len + pos;
  auto bin = [&](int m) {
    const float2 v = bb[(int64_t)m * len];
    return F2{v.x, v.y};
  };
  const int h = (M - 1) / 2;
  const F2 b0 = bin(0);
  const F2 bh = (M % 2 == 0) ? bin(M / 2) : F2{0.f, 0.f};
  F2 ev[kMaxM / 2], od[kMaxM / 2];
#pragma unroll
  for (int m = 1; m <= kMaxM / 2; ++m) {
    if (m > h) break;
    const F2 u = bin(m), v = bin(M - m);
    ev[m - 1] = f2_add(u, v);
    od[m - 1] = f2_add(u, f2_neg(v));
  }
  cd* out = a.pz[z] + (int64_t)fc * a.ns * len + pos;
  cdf* outf = a.pzf[z] + (int64_t)fc * a.ns * len + pos;
  for (int s = 0; s < a.ns; ++s) {
    F2 re = f2_add(b0, (s & 1) ? f2_neg(bh) : bh), im = {0.f, 0.f};
    int k = 0;
#pragma unroll
    for (int m = 1; m <= kMaxM / 2; ++m) {
      if (m > h) break;
      k += s;
      if (k >= M) k -= M;
      if (!CBP_CHECK(k >= 0 && k < M, 1)) k = 0;
      f2_mac(re, ev[m - 1], cs[k]);
      f2_mac(im, f2_neg(od[m - 1]), sn[k]);
    }
    re = f2_norm(re);
    im = f2_norm(im);
    outf[(int64_t)s * len] = cdf{re.hi, re.lo, im.hi, im.lo};
    if (a.pz_all || s == 0 || 2 * s == M)
      out[(int64_t)s * len] = mk((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo);
  }
}

}  // namespace

void launch_fold_dft(const Plan& p, char* ws, cudaStream_t st) {
  FoldDftArgs a;
  int maxlen = 0;
  for (int k = 0; k < 2; ++k) {
    a.bins[k] = ws + p.off_fbr[k];
    a.bins[2 + k] = ws + p.off_fbc[k];
    a.pz[k] = (cd*)(ws + p.off_pz2[k]);
    a.pz[2 + k] = (cd*)(ws + p.off_pz1[k]);
    a.pzf[k] = p.mixed ? (cdf*)(ws + p.off_pz2f[k]) : nullptr;
    a.pzf[2 + k] = p.mixed ? (cdf*)(ws + p.off_pz1f[k]) : nullptr;
  }
  a.len[0] = p.H1;
  a.len[1] = p.H2;
  a.len[2] = p.W1;
  a.len[3] = p.W2;
  for (int k = 0; k < 4; ++k) maxlen = a.len[k] > maxlen ? a.len[k] : maxlen;
  a.M = p.M;
  a.ns = p.ns;
  a.pz_all = p.pz_all;
  a.accepted = p.learned ? (const int*)(ws + p.off_acc) : nullptr;
  a.C = p.C;
  dim3 g((maxlen + kDftThreads - 1) / kDftThreads, p.n * p.C, 4);
  // bins of float32 frames are (hi, lo) pairs; the mixed path of float32
  // frames takes the float-float kernel
  if (!p.frames_f64 && p.mixed) k_fold_dft_ff<<<g, kDftThreads, 0, st>>>(a);
  else if (!p.frames_f64) k_fold_dft<true><<<g, kDftThreads, 0, st>>>(a);
  else k_fold_dft<false><<<g, kDftThreads, 0, st>>>(a);
}

void launch_eval(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                 cudaStream_t st) {
  launch_row_pass(p, b1, b2, ws, st, true, false);
  launch_fold_dft(p, ws, st);
}

}  // namespace cbp
