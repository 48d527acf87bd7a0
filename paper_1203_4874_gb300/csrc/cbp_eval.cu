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
// so the bins -- and the samples, whose M-point DFT runs in double -- carry
// ~1e-14 relative error on both paths; the mixed path also keeps float-float
// (hi + lo) copies for its extended-precision Gram on the float units.
#include "cbp_common.cuh"
#include "cbp_internal.h"

namespace cbp {
namespace {

constexpr int kDftThreads = 128;

struct FoldDftArgs {
  const double* bins[4];   // [pass * 2 + frame]; pass 0: row bins, 1: column bins; [n C][M][len]
  cd* pz[4];               // [n C][ns][len] samples
  cdf* pzf[4];             // float-float copies (mixed path) or null
  int len[4];
  int M, ns;
};

// M-point DFT of each position's M real bins, samples s < ns, using the
// symmetry of the roots: with e_m = b_m + b_(M-m), o_m = b_m - b_(M-m),
//   P_s = b_0 + sum_{m=1..(M-1)/2} (e_m cos(2 pi s m / M) - i o_m sin(2 pi s m / M))
//         [+ (-1)^s b_(M/2) when M is even].
__global__ void __launch_bounds__(kDftThreads) k_fold_dft(FoldDftArgs a) {
  __shared__ double cs[kMaxM], sn[kMaxM];
  for (int k = threadIdx.x; k < a.M; k += blockDim.x) sincospi(2.0 * (double)k / (double)a.M, &sn[k], &cs[k]);
  __syncthreads();
  const int z = blockIdx.z, fc = blockIdx.y, M = a.M, len = a.len[z];
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= len) return;
  const double* b = a.bins[z] + (int64_t)fc * M * len + pos;
  const int h = (M - 1) / 2;
  const double b0 = b[0];
  const double bh = (M % 2 == 0) ? b[(int64_t)(M / 2) * len] : 0.0;
  double ev[kMaxM / 2], od[kMaxM / 2];
#pragma unroll
  for (int m = 1; m <= kMaxM / 2; ++m) {
    if (m > h) break;
    const double u = b[(int64_t)m * len], v = b[(int64_t)(M - m) * len];
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
      re = fma(ev[m - 1], cs[k], re);
      im = fma(-od[m - 1], sn[k], im);
    }
    const cd pv = mk(re, im);
    out[(int64_t)s * len] = pv;
    if (outf) outf[(int64_t)s * len] = to_cdf(pv);
  }
}

}  // namespace

void launch_fold_dft(const Plan& p, char* ws, cudaStream_t st) {
  FoldDftArgs a;
  int maxlen = 0;
  for (int k = 0; k < 2; ++k) {
    a.bins[k] = (const double*)(ws + p.off_fbr[k]);
    a.bins[2 + k] = (const double*)(ws + p.off_fbc[k]);
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
  dim3 g((maxlen + kDftThreads - 1) / kDftThreads, p.n * p.C, 4);
  k_fold_dft<<<g, kDftThreads, 0, st>>>(a);
}

void launch_eval(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                 cudaStream_t st) {
  launch_row_pass(p, b1, b2, ws, st, true, false);
  launch_fold_dft(p, ws, st);
}

}  // namespace cbp
