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
// Mixed path: bins and samples in float, plus the z = 1 sample (s = 0) as the
// double-precision sum of the float bins, kept separately (it is real).
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
  void* pz[2];        // cpx<T> [n][C][ns][len_k]
  double* dc[2];      // optional, [n][C][len_k]
  int* bad;           // [n]
};

// One warp per row.  Lane l (l < g*M, g = floor(32/M)) owns bin m = l mod M
// and block-group q = l / M; at step k it reads column (k*g + q)*M + m, so
// the warp reads g*M consecutive elements per step.
template <typename T>
__global__ void __launch_bounds__(kRowWarps * 32)
k_eval_rows(FrameDesc f1, FrameDesc f2, int M, int ns, EvalOut out) {
  __shared__ cd wtab[kMaxM];
  __shared__ T bins[kRowWarps][32];
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
  const void* fb = frame_base(fr, f);
  const int64_t base = (int64_t)ch * fr.cs + (int64_t)r * fr.rs;
  T acc = 0;
  if (q < g) {
    for (int c = q * M + m; c < fr.w; c += g * M) acc += ld_frame<T>(fb, base + c, fr.f64);
  }
  bins[warp][lane] = acc;
  __syncwarp();
  if (lane < M) {
    T s = 0;
    for (int qq = 0; qq < g; ++qq) s += bins[warp][qq * M + lane];
    bins[warp][lane] = s;   // each lane only rewrites its own slot after reading
  }
  __syncwarp();
  if (lane < ns) {
    cpx<T> p = mk<T>(0, 0);
    for (int mm = 0; mm < M; ++mm) {
      cd w = wtab[(lane * mm) % M];
      T b = bins[warp][mm];
      p.re += b * (T)w.re;
      p.im += b * (T)w.im;
    }
    cpx<T>* dst = (cpx<T>*)out.pz[blockIdx.z];
    dst[((int64_t)fc * ns + lane) * fr.h + r] = p;
  }
  if (out.dc[blockIdx.z] && lane == 0) {
    double s = 0;
    for (int mm = 0; mm < M; ++mm) s += (double)bins[warp][mm];
    out.dc[blockIdx.z][(int64_t)fc * fr.h + r] = s;
  }
}

// One thread per column.  Bin m sums rows m, m + M, m + 2M, ...; a warp reads
// 32 consecutive columns of one row per step.  Also flags non-finite input.
template <typename T>
__global__ void __launch_bounds__(kColThreads)
k_eval_cols(FrameDesc f1, FrameDesc f2, int M, int ns, EvalOut out) {
  __shared__ cd wtab[kMaxM];
  __shared__ T bins[kMaxM][kColThreads];
  root_table(wtab, M);
  __syncthreads();
  const FrameDesc& fr = blockIdx.z ? f2 : f1;
  const int fc = blockIdx.y;
  const int f = fc / fr.c, ch = fc % fr.c;
  const int col = blockIdx.x * kColThreads + threadIdx.x;
  if (blockIdx.x * kColThreads >= fr.w) return;   // uniform per block
  const bool active = col < fr.w;
  const void* fb = frame_base(fr, f);
  const int64_t base = (int64_t)ch * fr.cs + col;
  bool finite = true;
  for (int m = 0; m < M; ++m) {
    T acc = 0;
    if (active) {
      int r = m;
      for (; r + 3 * M < fr.h; r += 4 * M) {
        T a0 = ld_frame<T>(fb, base + (int64_t)r * fr.rs, fr.f64);
        T a1 = ld_frame<T>(fb, base + (int64_t)(r + M) * fr.rs, fr.f64);
        T a2 = ld_frame<T>(fb, base + (int64_t)(r + 2 * M) * fr.rs, fr.f64);
        T a3 = ld_frame<T>(fb, base + (int64_t)(r + 3 * M) * fr.rs, fr.f64);
        acc += (a0 + a1) + (a2 + a3);
      }
      for (; r < fr.h; r += M) acc += ld_frame<T>(fb, base + (int64_t)r * fr.rs, fr.f64);
      finite = finite && isfinite(acc);
    }
    bins[m][threadIdx.x] = acc;
  }
  if (!finite) atomicOr(out.bad + f, 1);
  if (!active) return;
  cpx<T>* dst = (cpx<T>*)out.pz[blockIdx.z];
  for (int s = 0; s < ns; ++s) {
    cpx<T> p = mk<T>(0, 0);
    for (int mm = 0; mm < M; ++mm) {
      cd w = wtab[(s * mm) % M];
      T b = bins[mm][threadIdx.x];
      p.re += b * (T)w.re;
      p.im += b * (T)w.im;
    }
    dst[((int64_t)fc * ns + s) * fr.w + col] = p;
  }
  if (out.dc[blockIdx.z]) {
    double s = 0;
    for (int mm = 0; mm < M; ++mm) s += (double)bins[mm][threadIdx.x];
    out.dc[blockIdx.z][(int64_t)fc * fr.w + col] = s;
  }
}

}  // namespace

void launch_eval(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                 cudaStream_t st) {
  EvalOut rows, cols;
  for (int k = 0; k < 2; ++k) {
    rows.pz[k] = ws + p.off_pz2[k];
    cols.pz[k] = ws + p.off_pz1[k];
    rows.dc[k] = p.mixed ? (double*)(ws + p.off_dcz2[k]) : nullptr;
    cols.dc[k] = p.mixed ? (double*)(ws + p.off_dcz1[k]) : nullptr;
  }
  rows.bad = cols.bad = (int*)(ws + p.off_bad);
  const int hmax = b1.h > b2.h ? b1.h : b2.h;
  const int wmax = b1.w > b2.w ? b1.w : b2.w;
  dim3 gr((hmax + kRowWarps - 1) / kRowWarps, p.n * p.C, 2);
  dim3 gc((wmax + kColThreads - 1) / kColThreads, p.n * p.C, 2);
  if (p.mixed) {
    k_eval_rows<float><<<gr, kRowWarps * 32, 0, st>>>(b1, b2, p.M, p.ns, rows);
    k_eval_cols<float><<<gc, kColThreads, 0, st>>>(b1, b2, p.M, p.ns, cols);
  } else {
    k_eval_rows<double><<<gr, kRowWarps * 32, 0, st>>>(b1, b2, p.M, p.ns, rows);
    k_eval_cols<double><<<gc, kColThreads, 0, st>>>(b1, b2, p.M, p.ns, cols);
  }
}

}  // namespace cbp
