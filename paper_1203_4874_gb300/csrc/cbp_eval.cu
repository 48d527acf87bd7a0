// A1: evaluation of both blurred frames' bivariate z-polynomials at the M-th
// roots of unity, in both orders (Eq. 3; Section 5, "polynomial evaluation").
//
//   z2 = w^s  (rows kept):     P_Z2[s][r] = sum_c B[r][c] w^(s c)
//   z1 = w^s  (columns kept):  P_Z1[s][c] = sum_r B[r][c] w^(s r),   w = exp(-2 pi i / M)
//
// Because w^(s c) depends only on c mod M, each row (column) is first folded
// into M bins -- F2[r][m] = sum_{c = m mod M} B[r][c] -- and the M-point DFT
// of the bins gives every sample.  The frame is read once per direction,
// coalesced; only samples s <= M/2 are produced (real input: sample M - s is
// the conjugate of sample s).  The paper's own kernel (Section 5, one thread
// block per row/column, one shared-memory reduction per sample) re-reads the
// frame once per sample; the fold makes the cost independent of M.
//
// Float32 frames are folded with an exact float TwoSum accumulation (hi + lo),
// so the bins -- and the samples, whose M-point DFT runs in double -- carry
// ~1e-14 relative error on both paths; the mixed path also keeps float-float
// (hi + lo) copies for its extended-precision Gram on the float units.
#include "cbp_common.cuh"
#include "cbp_internal.h"

namespace cbp {
namespace {

constexpr int kRowWarps = 8;
constexpr int kColThreads = 128;

__device__ __forceinline__ void root_table(cd* tab, int M) {
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)M, &s, &c);
    tab[k] = mk(c, s);
  }
}

struct EvalOut {
  cd* pz[2];          // [n][C][ns][len_k] double samples
  cdf* pzf[2];        // optional float-float copies (mixed path)
  int* bad;           // [n]
};

// Running sum of float terms kept exactly as hi + lo (Knuth's TwoSum), so a
// fold of float32 frames is accurate to ~1e-14 using float arithmetic only.
struct TwoSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = hi + x;
    const float z = t - hi;
    lo += (hi - (t - z)) + (x - z);
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
struct DoubleSum {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};

// M-point DFT of double bins b[0..M) at sample s: sum_m b[m] w^(s m).
__device__ __forceinline__ cd bins_dft(const double* b, int bstride, const cd* wtab, int M, int s) {
  cd p = mk(0.0, 0.0);
  int e = 0;
  for (int mm = 0; mm < M; ++mm) {
    const double v = b[mm * bstride];
    p.re += v * wtab[e].re;
    p.im += v * wtab[e].im;
    e += s;
    if (e >= M) e -= M;
  }
  return p;
}

// One warp per row.  Lane l (l < g*M, g = floor(32/M)) owns bin m = l mod M
// and block-group q = l / M; at step k it reads column (k*g + q)*M + m, so
// the warp reads g*M consecutive elements per step.
template <typename Acc, typename In>
__global__ void __launch_bounds__(kRowWarps * 32)
k_eval_rows(FrameDesc f1, FrameDesc f2, int M, int ns, EvalOut out) {
  __shared__ cd wtab[kMaxM];
  __shared__ double bins[kRowWarps][32];
  root_table(wtab, M);
  __syncthreads();
  const FrameDesc& fr = blockIdx.z ? f2 : f1;
  const int fc = blockIdx.y;                 // frame * C + channel
  const int f = fc / fr.c, ch = fc % fr.c;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * kRowWarps + warp;
  if (r >= fr.h) return;                     // whole warp leaves together
  const int g = 32 / M;
  const int m = lane % M, q = lane / M;
  const In* row = (const In*)frame_base(fr, f) + (int64_t)ch * fr.cs + (int64_t)r * fr.rs;
  Acc acc;
  if (q < g)
    for (int c = q * M + m; c < fr.w; c += g * M) acc.add(__ldg(row + c));
  bins[warp][lane] = acc.value();
  __syncwarp();
  if (lane < M) {
    double v = 0;
    for (int qq = 0; qq < g; ++qq) v += bins[warp][qq * M + lane];
    bins[warp][lane] = v;   // each lane only rewrites its own slot after reading
  }
  __syncwarp();
  if (lane < ns) {
    const cd pv = bins_dft(&bins[warp][0], 1, wtab, M, lane);
    const int64_t o = ((int64_t)fc * ns + lane) * fr.h + r;
    out.pz[blockIdx.z][o] = pv;
    if (out.pzf[blockIdx.z]) out.pzf[blockIdx.z][o] = to_cdf(pv);
  }
}

// One thread per column.  Bin m sums rows m, m + M, m + 2M, ...; a warp reads
// 32 consecutive columns of one row per step.  Also flags non-finite input.
template <typename Acc, typename In>
__global__ void __launch_bounds__(kColThreads)
k_eval_cols(FrameDesc f1, FrameDesc f2, int M, int ns, EvalOut out) {
  __shared__ cd wtab[kMaxM];
  __shared__ double bins[kMaxM][kColThreads];
  root_table(wtab, M);
  __syncthreads();
  const FrameDesc& fr = blockIdx.z ? f2 : f1;
  const int fc = blockIdx.y;
  const int f = fc / fr.c, ch = fc % fr.c;
  const int col = blockIdx.x * kColThreads + threadIdx.x;
  if (blockIdx.x * kColThreads >= fr.w) return;   // uniform per block
  const bool active = col < fr.w;
  const In* base = (const In*)frame_base(fr, f) + (int64_t)ch * fr.cs + col;
  bool finite = true;
  for (int m = 0; m < M; ++m) {
    Acc acc;
    if (active) {
      int r = m;
      for (; r + 3 * M < fr.h; r += 4 * M) {
        const In a0 = __ldg(base + (int64_t)r * fr.rs);
        const In a1 = __ldg(base + (int64_t)(r + M) * fr.rs);
        const In a2 = __ldg(base + (int64_t)(r + 2 * M) * fr.rs);
        const In a3 = __ldg(base + (int64_t)(r + 3 * M) * fr.rs);
        acc.add(a0);
        acc.add(a1);
        acc.add(a2);
        acc.add(a3);
      }
      for (; r < fr.h; r += M) acc.add(__ldg(base + (int64_t)r * fr.rs));
      finite = finite && isfinite(acc.value());
    }
    bins[m][threadIdx.x] = acc.value();
  }
  if (!finite) atomicOr(out.bad + f, 1);
  if (!active) return;
  for (int s = 0; s < ns; ++s) {
    const cd pv = bins_dft(&bins[0][threadIdx.x], kColThreads, wtab, M, s);
    const int64_t o = ((int64_t)fc * ns + s) * fr.w + col;
    out.pz[blockIdx.z][o] = pv;
    if (out.pzf[blockIdx.z]) out.pzf[blockIdx.z][o] = to_cdf(pv);
  }
}

}  // namespace

void launch_eval(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                 cudaStream_t st) {
  EvalOut rows, cols;
  for (int k = 0; k < 2; ++k) {
    rows.pz[k] = (cd*)(ws + p.off_pz2[k]);
    cols.pz[k] = (cd*)(ws + p.off_pz1[k]);
    rows.pzf[k] = p.mixed ? (cdf*)(ws + p.off_pz2f[k]) : nullptr;
    cols.pzf[k] = p.mixed ? (cdf*)(ws + p.off_pz1f[k]) : nullptr;
  }
  rows.bad = cols.bad = (int*)(ws + p.off_bad);
  const int hmax = b1.h > b2.h ? b1.h : b2.h;
  const int wmax = b1.w > b2.w ? b1.w : b2.w;
  dim3 gr((hmax + kRowWarps - 1) / kRowWarps, p.n * p.C, 2);
  dim3 gc((wmax + kColThreads - 1) / kColThreads, p.n * p.C, 2);
  if (b1.f64) {   // double frames: double sums
    k_eval_rows<DoubleSum, double><<<gr, kRowWarps * 32, 0, st>>>(b1, b2, p.M, p.ns, rows);
    k_eval_cols<DoubleSum, double><<<gc, kColThreads, 0, st>>>(b1, b2, p.M, p.ns, cols);
  } else {        // float frames: exact float TwoSum accumulation
    k_eval_rows<TwoSum, float><<<gr, kRowWarps * 32, 0, st>>>(b1, b2, p.M, p.ns, rows);
    k_eval_cols<TwoSum, float><<<gc, kColThreads, 0, st>>>(b1, b2, p.M, p.ns, cols);
  }
}

}  // namespace cbp
