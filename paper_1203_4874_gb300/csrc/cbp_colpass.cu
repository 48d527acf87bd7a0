// A6, the column pass of the dual-kernel Fourier deconvolution, fused with the
// kernel spectra, for grids whose column length Ph = N1 N2 splits into two
// factors that one thread can transform in registers (the 1080p grid:
// 1120 = 32 x 35).
//
// For one strip of four spectrum columns v of one frame channel:
//   B^_k(., v)  column DFTs of both frames' row spectra (rows >= H_k are zero),
//   K^_k(., v)  the kernels' spectra, from their row transforms
//               R_k,p(v) = sum_q K_k[p][q] w_Pw^(q v)  (p < t_k),
//   I^ = (conj(K^1) B^1 + conj(K^2) B^2) / (|K^1|^2 + |K^2|^2 + eps),
//   inverse column DFT of I^, rows < H written out.
// The transforms are the two-factor (Cooley-Tukey) split of a length-N1 N2
// DFT, with n = n1 + N1 n2 and u = k2 + N2 k1:
//   X[k2 + N2 k1] = sum_n1 w_N1^(n1 k1) w_Ph^(n1 k2) sum_n2 x[n1 + N1 n2] w_N2^(n2 k2).
// Step 1: one task per (n1, column) loads its N2 rows from HBM, transforms
// them in registers, applies the twiddles and leaves them in shared memory.
// Step 2: one task per (k2, column) reads its N1 values, transforms them in
// registers, and holds the N1 output rows u = k2 + N2 k1 of that column: both
// frames' spectra, both kernels' spectra (an N1-point DFT of the t_k nonzero
// terms R_k,p w_Ph^(p k2)), the formula, and the first half of the inverse
// transform all happen there; step 3 (one task per (n1, column)) finishes the
// inverse and writes the rows < H.  Two block barriers per channel strip; the
// kernel spectra never touch HBM.
#include "cbp_common.cuh"
#include "cbp_dft.cuh"
#include "cbp_internal.h"

namespace cbp {
namespace {

constexpr int kFcThreads = 160;
constexpr int kFcCols = 4;          // spectrum columns per strip (one 32-byte sector per row)
constexpr int kFcMaxT = 32;         // kernel rows the row-transform table holds

struct FusedColArgs {
  const cf* spec[2];   // [n][C][H_k][Pw2p] row spectra of B1, B2
  cf* ihat;            // [n][C][H][Pw2p] deconvolved spectrum (column-inverse done)
  const double* kd;    // [n][t1 t1 + t2 t2] kernels
  const cf* tw_h;      // w_Ph^k, k < Ph
  const cf* tw_w;      // w_Pw^k, k < Pw
  int H1, H2, H, C, t1, t2, Pw, Pw2, Pw2p;
  float eps;
};

// Shared memory: two frames' buffers of N2 slot rows of (N1 + 1) slots (the
// pad spreads step 2's strided reads over the banks), kFcCols columns per
// slot, and the kernels' row transforms.
template <int N1, int N2>
struct FcSmem {
  static constexpr int kPitch = N1 + 1;
  static constexpr int kSlots = kPitch * N2;
  static constexpr size_t kBuf = (size_t)kSlots * kFcCols;          // cf per frame buffer
  static constexpr size_t kBytes = (2 * kBuf + 2 * (size_t)kFcMaxT * kFcCols) * sizeof(cf);
};

__device__ __forceinline__ cf ldg_cf(const cf* p) {
  const float2 v = __ldg((const float2*)p);
  return mk(v.x, v.y);
}

template <int N1, int N2>
__global__ void __launch_bounds__(kFcThreads, 3) k_col_deconv_fused(FusedColArgs a) {
  using L = FcSmem<N1, N2>;
  constexpr int P = L::kPitch;
  constexpr int Ph = N1 * N2;
  extern __shared__ __align__(16) char smem[];
  cf* buf0 = (cf*)smem;
  cf* buf1 = buf0 + L::kBuf;
  cf* rt = buf1 + L::kBuf;                 // [2][kFcMaxT][kFcCols] kernel row transforms
  const int fc = blockIdx.y, f = fc / a.C;
  const int v0 = blockIdx.x * kFcCols;
  const int tid = threadIdx.x;

  // kernel row transforms R_k,p(v) for the strip's columns (zero past Pw2)
  const double* K1 = a.kd + (int64_t)f * (a.t1 * a.t1 + a.t2 * a.t2);
  for (int e = tid; e < 2 * kFcMaxT * kFcCols; e += kFcThreads) {
    const int k = e / (kFcMaxT * kFcCols), p = (e / kFcCols) % kFcMaxT, col = e % kFcCols;
    const int t = k ? a.t2 : a.t1, v = v0 + col;
    const double* K = K1 + (k ? a.t1 * a.t1 : 0) + p * t;
    cf acc = mk(0.f, 0.f);
    if (p < t && v < a.Pw2) {
      int w = 0;                                   // (q v) mod Pw, incrementally
      for (int q = 0; q < t; ++q) {
        acc = acc + (float)K[q] * ldg_cf(a.tw_w + w);
        w += v;
        if (w >= a.Pw) w -= a.Pw;
      }
    }
    rt[e] = acc;
  }

  // ---- step 1: N2-point DFTs down the columns, twiddled, into shared memory
  for (int task = tid; task < 2 * N1 * kFcCols; task += kFcThreads) {
    const int fr = task / (N1 * kFcCols), r = task % (N1 * kFcCols);
    const int n1 = r / kFcCols, col = r % kFcCols;
    const int Hk = fr ? a.H2 : a.H1;
    const bool cv = v0 + col < a.Pw2;
    const cf* src = a.spec[fr] + ((int64_t)fc * Hk) * a.Pw2p + v0 + col;
    cf x[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const int row = n1 + N1 * n2;
      x[n2] = (cv && row < Hk) ? ldg_cf(src + (int64_t)row * a.Pw2p) : mk(0.f, 0.f);
    }
    reg_dft<false, N2>(x);
    cf* dst = (fr ? buf1 : buf0) + n1 * kFcCols + col;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      cf y = x[reg_pos<N2>(k2)];
      if (k2) y = y * ldg_cf(a.tw_h + n1 * k2);      // w_Ph^(n1 k2), n1 k2 < Ph
      dst[k2 * P * kFcCols] = y;
    }
  }
  __syncthreads();

  // ---- step 2: N1-point DFTs across, the formula, the inverse N1-point DFTs
  if (tid < N2 * kFcCols) {
    const int k2 = tid / kFcCols, col = tid % kFcCols;
    cf* s0 = buf0 + (k2 * P) * kFcCols + col;      // slot (j, k2) at s[j * kFcCols]
    cf* s1 = buf1 + (k2 * P) * kFcCols + col;
    // both frames' column spectra at rows u = k2 + N2 k1, back into their slots
    {
      cf x[N1];
#pragma unroll
      for (int j = 0; j < N1; ++j) x[j] = s1[j * kFcCols];
      reg_dft<false, N1>(x);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) s1[k1 * kFcCols] = x[reg_pos<N1>(k1)];
    }
    {
      cf x[N1];
#pragma unroll
      for (int j = 0; j < N1; ++j) x[j] = s0[j * kFcCols];
      reg_dft<false, N1>(x);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) s0[k1 * kFcCols] = x[reg_pos<N1>(k1)];
    }
    // kernel spectra at the same rows: K^(k2 + N2 k1) = DFT_N1 over p of R_p w_Ph^(p k2)
    const cf* r1 = rt + col;
    const cf* r2 = rt + kFcMaxT * kFcCols + col;
    float d1[N1];
    {
      cf kh[N1];
#pragma unroll
      for (int p = 0; p < N1; ++p) {
        kh[p] = mk(0.f, 0.f);
        if (p < a.t1) kh[p] = p ? r1[p * kFcCols] * ldg_cf(a.tw_h + p * k2) : r1[0];
      }
      reg_dft<false, N1>(kh);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const cf k = kh[reg_pos<N1>(k1)];
        s0[k1 * kFcCols] = cmulc(k, s0[k1 * kFcCols]);    // conj(K^1) B^1
        d1[k1] = abs2(k);
      }
    }
    cf iv[N1];
    {
      cf kh[N1];
#pragma unroll
      for (int p = 0; p < N1; ++p) {
        kh[p] = mk(0.f, 0.f);
        if (p < a.t2) kh[p] = p ? r2[p * kFcCols] * ldg_cf(a.tw_h + p * k2) : r2[0];
      }
      reg_dft<false, N1>(kh);
      const float eps = a.eps;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const cf k = kh[reg_pos<N1>(k1)];
        const cf num = s0[k1 * kFcCols] + cmulc(k, s1[k1 * kFcCols]);
        const float den = d1[k1] + abs2(k) + eps;
        iv[k1] = (den != 0.f ? __frcp_rn(den) : 0.f) * num;
      }
    }
    // inverse over k1, twiddled by w_Ph^(-n1 k2), into this task's slots
    reg_dft<true, N1>(iv);
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
      cf z = iv[reg_pos<N1>(n1)];
      if (n1 && k2) z = z * conj(ldg_cf(a.tw_h + n1 * k2));
      s0[n1 * kFcCols] = z;
    }
  }
  __syncthreads();

  // ---- step 3: inverse N2-point DFTs down the columns, rows < H out
  if (tid < N1 * kFcCols) {
    const int n1 = tid / kFcCols, col = tid % kFcCols;
    const cf* src = buf0 + n1 * kFcCols + col;
    cf x[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) x[k2] = src[k2 * P * kFcCols];
    reg_dft<true, N2>(x);
    if (v0 + col < a.Pw2) {
      cf* dst = a.ihat + ((int64_t)fc * a.H) * a.Pw2p + v0 + col;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int row = n1 + N1 * n2;
        if (row < a.H) dst[(int64_t)row * a.Pw2p] = x[reg_pos<N2>(n2)];
      }
    }
  }
  static_assert(N1 <= kFcMaxT, "kernel rows beyond the row-transform table");
  static_assert(Ph == N1 * N2, "");
}

template <int N1, int N2>
void run_fused(const Plan& p, char* ws, cudaStream_t st) {
  FusedColArgs a;
  a.spec[0] = (const cf*)(ws + p.off_spec[0]);
  a.spec[1] = (const cf*)(ws + p.off_spec[1]);
  a.ihat = (cf*)(ws + p.off_ihat);
  a.kd = (const double*)(ws + p.off_kd);
  a.tw_h = (const cf*)(ws + p.off_tw_h);
  a.tw_w = (const cf*)(ws + p.off_tw_w);
  a.H1 = p.H1;
  a.H2 = p.H2;
  a.H = p.H;
  a.C = p.C;
  a.t1 = p.t1;
  a.t2 = p.t2;
  a.Pw = p.Pw;
  a.Pw2 = p.Pw2;
  a.Pw2p = p.Pw2p;
  a.eps = (float)p.eps;
  const size_t sm = FcSmem<N1, N2>::kBytes;
  cudaFuncSetAttribute(k_col_deconv_fused<N1, N2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_col_deconv_fused<N1, N2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  dim3 g((p.Pw2 + kFcCols - 1) / kFcCols, p.n * p.C);
  k_col_deconv_fused<N1, N2><<<g, kFcThreads, sm, st>>>(a);
}

}  // namespace

bool col_pass_fused(const Plan& p) {
  if (p.fft_f64 || p.single_kernel) return false;
  if (p.t1 > kFcMaxT || p.t2 > kFcMaxT) return false;
  return p.Ph == 1120 && p.t1 <= 32 && p.t2 <= 32;
}

void launch_col_deconv_fused(const Plan& p, char* ws, cudaStream_t st) {
  run_fused<32, 35>(p, ws, st);
}

}  // namespace cbp
