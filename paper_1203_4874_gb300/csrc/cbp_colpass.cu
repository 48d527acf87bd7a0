// A6, the column pass of the dual-kernel Fourier deconvolution, fused with the
// kernel spectra, for grids whose column length Ph = N1 N2 splits into two
// factors that one thread can transform in registers (the 1080p grid:
// 1120 = 32 x 35).
//
// For one strip of four spectrum columns v of one frame channel:
//   B^_k(., v)  column DFTs of both frames' row spectra (rows >= H_k are zero),
//   K^_k(., v)  the kernels' spectra, from their row transforms
//               R_k,p(v) = sum_q K_k[p][q] w_Pw^(q v)  (p < t_k; made once per
//               pair by k_kernel_rows and shared by the pair's channels),
//   I^ = (conj(K^1) B^1 + conj(K^2) B^2) / (|K^1|^2 + |K^2|^2 + eps),
//   inverse column DFT of I^, rows < H written out.
// The transforms are the two-factor (Cooley-Tukey) split of a length-N1 N2
// DFT, with n = n1 + N1 n2 and u = k2 + N2 k1:
//   X[k2 + N2 k1] = sum_n1 w_N1^(n1 k1) w_Ph^(n1 k2) sum_n2 x[n1 + N1 n2] w_N2^(n2 k2).
// Both frames' strips and the strip's row transforms are staged in shared
// memory (cp.async) first.
// Step 1: one task per (n1, column) takes its N2 rows, transforms them in
// registers, applies the twiddles and puts them back in place.
// Step 2: one task per (k2, column) reads its N1 values, transforms them in
// registers, and holds the N1 output rows u = k2 + N2 k1 of that column: both
// frames' spectra, both kernels' spectra (an N1-point DFT of the t_k nonzero
// terms R_k,p w_Ph^(p k2)), the formula, and the first half of the inverse
// transform all happen there; step 3 (one task per (n1, column)) finishes the
// inverse and writes the rows < H.  Two block barriers per channel strip; the
// kernel spectra never touch HBM.
#include <algorithm>
#include "cbp_common.cuh"
#include "cbp_dft.cuh"
#include "cbp_internal.h"
#ifdef CBP_PHASE_TIMING
#include <cstdio>
#define FC_TICK(i) \
  do {             \
    if (threadIdx.x == 0) tck[i] = clock64(); \
  } while (0)
#else
#define FC_TICK(i) \
  do {             \
  } while (0)
#endif

namespace cbp {

CBP_CHECKS_TU(kChkColpass)

namespace {

constexpr int kFcThreads = 160;
#ifndef CBP_FC_MIN_BLOCKS
#define CBP_FC_MIN_BLOCKS 3   // resident blocks per SM the register budget is set for
#endif
constexpr int kFcCols = 4;          // spectrum columns per strip (one 32-byte sector per row)
constexpr int kFcMaxT = 32;         // kernel rows the row-transform table holds

struct FusedColArgs {
  const cf* spec[2];   // [n][C][H_k][Pw2p] row spectra of B1, B2
  cf* ihat;            // [n][C][H][Pw2p] deconvolved spectrum (column-inverse done)
  const cf* krow;      // [n][2][max(t1, t2)][Pw2p] kernels' row transforms (k_kernel_rows)
  const cf* tw1;       // w_Ph^(n1 m) at [m][n1] (step 1)
  const cf* tw2;       // w_Ph^(p k2) at [p][k2] (step 2: kernel spectra, inverse)
  const int* accepted; // learned path: pairs whose proposal passed the gate (or null)
  double* rpart;       // RESID: [n C][strips][2] residual sums
  int H1, H2, H, C, t1, t2, Pw, Pw2, Pw2p;
  float eps;
};

// Shared memory: both frames' column strips (Ph rows of kFcCols columns; row /
// slot s at physical row fc_phys(s)) and the kernels' row transforms.
template <int N1, int N2>
struct FcSmem {
  static constexpr size_t kBuf = (size_t)N1 * N2 * kFcCols;          // cf per frame buffer
  static constexpr size_t kBytes = (2 * kBuf + 2 * (size_t)kFcMaxT * kFcCols) * sizeof(cf);
};

// Logical slot s = j + N1 m (the strip's row index; step 1's task j = n1
// holds slots j + N1 m, step 2's task m = k2 holds slots j + N1 k2) lives at
// physical row s ^ (m & 3): step 2's lanes, eight values of m apart by N1
// rows, then fall on four different groups of eight banks (two wavefronts per
// 8-byte access, the minimum), and consecutive slots stay in one 4-row group.
template <int N1>
__device__ __forceinline__ int fc_phys(int s) {
  return s ^ ((s / N1) & 3);
}

__device__ __forceinline__ cf ldg_cf(const cf* p) {
  const float2 v = __ldg((const float2*)p);
  return mk(v.x, v.y);
}

__device__ __forceinline__ void fc_cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes)
               : "memory");
}

// Stage the strip's rows of one row spectrum (rows >= Hk and columns >= the
// strip's valid count zero-filled) into buf at the swizzled rows.
template <int N1, int N2>
__device__ __forceinline__ void fc_stage(cf* buf, const cf* src, int Hk, int Pw2p, int nv) {
  constexpr int Ph = N1 * N2;
  for (int e = threadIdx.x; e < Ph * 2; e += kFcThreads) {
    const int row = e >> 1, half = e & 1;
    const int valid = row < Hk ? max(0, min(2, nv - 2 * half)) * (int)sizeof(cf) : 0;
    const cf* g = valid ? src + (int64_t)row * Pw2p + 2 * half : src;
    if (CBP_CHECK(fc_phys<N1>(row) < Ph && 2 * half + 2 <= kFcCols, 0))
      fc_cp_async16(buf + fc_phys<N1>(row) * kFcCols + 2 * half, g, valid);
  }
}

// 1 / x by the hardware approximation (relative error below 2^-22; the
// formula's inputs carry single-precision FFT rounding already).
__device__ __forceinline__ float fc_rcp(float x) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The kernels' row transforms R_k,p(v) = sum_q K_k[p][q] w_Pw^(q v) of the
// half-spectrum columns v < Pw2 (zero on the padding up to Pw2p), once per
// pair: the column pass of each of its channels copies in the rows it needs.
constexpr int kKrThreads = 128;
__global__ void __launch_bounds__(kKrThreads) k_kernel_rows(const double* kd, const cf* tw_w, cf* krow,
                                                            int t1, int t2, int Pw, int Pw2,
                                                            int Pw2p) {
  const int v = blockIdx.x * kKrThreads + threadIdx.x;
  const int p = blockIdx.y, f = blockIdx.z >> 1, k = blockIdx.z & 1;
  const int t = k ? t2 : t1, tm = max(t1, t2);
  if (p >= t || v >= Pw2p) return;
  const double* K = kd + (int64_t)f * (t1 * t1 + t2 * t2) + (k ? t1 * t1 : 0) + p * t;
  cf acc = mk(0.f, 0.f);
  if (v < Pw2) {
    int w = 0;                                   // (q v) mod Pw, incrementally
    for (int q = 0; q < t; ++q) {
      acc = acc + (float)K[q] * ldg_cf(tw_w + w);
      w += v;
      if (w >= Pw) w -= Pw;
    }
  }
  if (CBP_CHECK(p < tm && v < Pw2p, 1)) krow[(((int64_t)f * 2 + k) * tm + p) * Pw2p + v] = acc;
}

// Inputs of an N1-point DFT giving a kernel's column spectrum K^(k2 + N2 k1):
// R_p w_Ph^(p k2) for its t nonzero rows p (r: the strip's row transforms of
// this column, stride kFcCols; tw: w_Ph^(p k2) at [p][k2], already offset by k2).
template <int N1, int N2>
__device__ __forceinline__ void fc_kspec_in(cf* v, const cf* r, int t, const cf* tw) {
#pragma unroll
  for (int p = 0; p < N1; ++p) {
    v[p] = mk(0.f, 0.f);
    if (p < t) v[p] = p ? r[p * kFcCols] * ldg_cf(tw + N2 * p) : r[0];
  }
}

// The formula's arithmetic spelled out with explicit rounding (no contraction
// left to the compiler), so that both variants of the pass round alike.
__device__ __forceinline__ cf fc_cmulc(cf k, cf b) {   // conj(k) b
  return mk(__fmaf_rn(k.re, b.re, __fmul_rn(k.im, b.im)), __fmaf_rn(k.re, b.im, -__fmul_rn(k.im, b.re)));
}
__device__ __forceinline__ float fc_abs2(cf k) { return __fmaf_rn(k.re, k.re, __fmul_rn(k.im, k.im)); }
// I^ = (t1 + conj(K2) B2) / (d1 + |K2|^2 + eps), t1 = conj(K1) B1, d1 = |K1|^2
__device__ __forceinline__ cf fc_formula(cf t1, float d1, cf k2, cf b2, float eps) {
  const cf t2 = fc_cmulc(k2, b2);
  const cf num = bf_add(t1, t2);                 // paired, rounded as two __fadd_rn
  const float den = __fadd_rn(__fadd_rn(d1, fc_abs2(k2)), eps);
  const float r = den != 0.f ? fc_rcp(den) : 0.f;
  return bf_scale(r, num);                       // paired, rounded as two __fmul_rn
}

// RESID (learned path): the same pass with the proposal's kernels, and besides
// the deconvolved spectrum the strip's part of the consistency residual,
//   sum |K2^ B1^ - K1^ B2^|^2 and sum |B1^|^2 over the strip's (u, v),
// each half-spectrum column counted twice except v = 0 and v = Pw/2 (its own
// mirror): by Parseval their ratio is rho^2 of the circular convolutions.  Both
// kernels' spectra are held in registers at once (two blocks per SM).
// Without RESID, pairs whose proposal was accepted are skipped.
template <int N1, int N2, bool RESID>
__global__ void __launch_bounds__(kFcThreads, RESID ? 2 : CBP_FC_MIN_BLOCKS)
k_col_deconv_fused(FusedColArgs a) {
  using L = FcSmem<N1, N2>;
  constexpr int Ph = N1 * N2;
  constexpr int S = kFcCols;                // slot stride (cf) in a buffer
  constexpr int B1 = (int)L::kBuf;          // buffer 1 relative to buffer 0 (cf)
  extern __shared__ __align__(16) char smem[];
  cf* buf0 = (cf*)smem;
  cf* rt = buf0 + 2 * L::kBuf;              // [2][kFcMaxT][kFcCols] kernel row transforms
  const int fc = blockIdx.y, f = fc / a.C;
  if (!RESID && a.accepted && a.accepted[f]) return;   // the proposal's pass stands
  const int v0 = blockIdx.x * kFcCols;
  const int nv = min(kFcCols, a.Pw2 - v0);
  const int tid = threadIdx.x;
#ifdef CBP_PHASE_TIMING
  long long tck[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#endif
  FC_TICK(0);

  // both frames' strips in flight while the kernels' row transforms are made
  fc_stage<N1, N2>(buf0, a.spec[0] + ((int64_t)fc * a.H1) * a.Pw2p + v0, a.H1, a.Pw2p, nv);
  fc_stage<N1, N2>(buf0 + B1, a.spec[1] + ((int64_t)fc * a.H2) * a.Pw2p + v0, a.H2, a.Pw2p, nv);
  asm volatile("cp.async.commit_group;\n" ::: "memory");

  // the kernels' row transforms R_k,p(v) of the strip's columns (rows p < t_k;
  // made once per pair by k_kernel_rows), copied in with the strips
  {
    const int tm = max(a.t1, a.t2);
    const cf* KR = a.krow + (int64_t)f * 2 * tm * a.Pw2p + v0;
    for (int e = tid; e < 2 * tm * 2; e += kFcThreads) {
      const int half = e & 1, kp = e >> 1, k = kp / tm, p = kp - k * tm;
      if (p < (k ? a.t2 : a.t1) && CBP_CHECK(p < kFcMaxT && v0 + 4 <= a.Pw2p, 2))
        fc_cp_async16(rt + (k * kFcMaxT + p) * kFcCols + 2 * half,
                      KR + ((int64_t)k * tm + p) * a.Pw2p + 2 * half, 16);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  FC_TICK(1);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  FC_TICK(2);

  // Slot (j, m) = logical row j + N1 m sits at physical row (j ^ (m & 3)) + N1 m
  // (fc_phys): with four base pointers per thread every access below is a
  // base plus an immediate offset.
  // Steps 1 and 3 share one code path (phase 0: forward N2-point DFTs of both
  // frames, twiddled, in place; phase 1: the inverse as conj(DFT(conj(.))), rows
  // < H out), with step 2 between them: one copy of each transform's code.
  // ---- step 1 (phase 0), step 2, step 3 (phase 1)
#pragma unroll 1
  for (int ph = 0; ph < 2; ++ph) {
    if (ph == 1) {
      __syncthreads();
      FC_TICK(3);
      // ---- step 2: N1-point DFTs across, the formula, the inverse N1-point DFTs
      float rn = 0.f, rd = 0.f;   // RESID: this task's residual sums
      if (tid < N2 * kFcCols) {
        const int k2 = tid / kFcCols, col = tid % kFcCols;
        (void)CBP_CHECK((N1 * k2 + N1) * S <= B1, 3);   // this task's slots inside the strip
        cf* q[4];
        {
          cf* base = buf0 + (N1 * k2) * S + col;
#pragma unroll
          for (int c = 0; c < 4; ++c) q[c] = base + (c ^ (k2 & 3)) * S;
        }
        // element j of this task's slots: q[j & 3][(j & ~3) S] (+ B1 for frame 2)
#define FC_AT(j) q[(j) & 3][((j) & ~3) * S]
#define FC_AT1(j) q[(j) & 3][((j) & ~3) * S + B1]
        float d1[N1];
        cf x[N1];          // the working transform; ends up holding I^ at reg_pos order
        cf y[N1];          // RESID: K^1 while K^2 is made
        const float eps = a.eps;
        // five N1-point DFTs through one code path: frame 2's and frame 1's
        // column spectra (back into their slots), the two kernels' spectra
        // K^(k2 + N2 k1) = DFT_N1 over p of R_p w_Ph^(p k2), each consumed by its
        // part of the formula at once, and the inverse (conjugated in and out)
#pragma unroll 1
        for (int it = 0; it < (RESID ? 2 : 5); ++it) {
          if (it == 0) {
#pragma unroll
            for (int j = 0; j < N1; ++j) x[j] = FC_AT1(j);
          } else if (it == 1 || it == 4) {
#pragma unroll
            for (int j = 0; j < N1; ++j) x[j] = FC_AT(j);
          } else {
            fc_kspec_in<N1, N2>(x, rt + (it - 2) * kFcMaxT * kFcCols + col, it == 2 ? a.t1 : a.t2,
                                a.tw2 + k2);
          }
          reg_dft<false, N1>(x);
          if (it == 0) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) FC_AT1(k1) = x[reg_pos<N1>(k1)];
          } else if (it == 1) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) FC_AT(k1) = x[reg_pos<N1>(k1)];
          } else if (it == 2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
              const cf k = x[reg_pos<N1>(k1)];
              FC_AT(k1) = fc_cmulc(k, FC_AT(k1));       // conj(K^1) B^1
              d1[k1] = fc_abs2(k);
            }
          } else if (it == 3) {
            // I^(k2 + N2 k1), conjugated, into this task's slots in natural
            // order: the inverse runs as conj(DFT(conj(.))) on the next pass
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) {
              const cf k = x[reg_pos<N1>(k1)];
              FC_AT(k1) = conj(fc_formula(FC_AT(k1), d1[k1], k, FC_AT1(k1), eps));
            }
          } else {
            // the inverse over k1, twiddled by w_Ph^(-n1 k2), into this task's slots
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) {
              cf z = conj(x[reg_pos<N1>(n1)]);
              if (n1) z = z * conj(ldg_cf(a.tw2 + N2 * n1 + k2));
              FC_AT(n1) = z;
            }
          }
        }
        if constexpr (RESID) {
          // both kernels' spectra at once (K^1 in y, K^2 in x), the residual sums
          // and the formula
          fc_kspec_in<N1, N2>(y, rt + col, a.t1, a.tw2 + k2);
          reg_dft<false, N1>(y);
          fc_kspec_in<N1, N2>(x, rt + kFcMaxT * kFcCols + col, a.t2, a.tw2 + k2);
          reg_dft<false, N1>(x);
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) {
            const cf kk1 = y[reg_pos<N1>(k1)], kk2 = x[reg_pos<N1>(k1)];
            const cf b1 = FC_AT(k1), b2 = FC_AT1(k1);
            const cf r = kk2 * b1 - kk1 * b2;
            rn += abs2(r);
            rd += abs2(b1);
            x[reg_pos<N1>(k1)] = fc_formula(fc_cmulc(kk1, b1), fc_abs2(kk1), kk2, b2, eps);
          }
        }
        if constexpr (RESID) {
          // inverse over k1, twiddled by w_Ph^(-n1 k2), into this task's slots
          cf iv[N1];
#pragma unroll
          for (int k1 = 0; k1 < N1; ++k1) iv[k1] = x[reg_pos<N1>(k1)];
          reg_dft<true, N1>(iv);
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) {
            cf z = iv[reg_pos<N1>(n1)];
            if (n1) z = z * conj(ldg_cf(a.tw2 + N2 * n1 + k2));
            FC_AT(n1) = z;
          }
        }
#undef FC_AT
#undef FC_AT1
      }
      if constexpr (RESID) {
        __shared__ double red[2][kFcThreads / 32];
        const int v = v0 + tid % kFcCols;
        const double wv = (v == 0 || 2 * v == a.Pw) ? 1.0 : 2.0;
        const double sn = warp_sum(wv * (double)rn), sd = warp_sum(wv * (double)rd);
        if ((tid & 31) == 0) {
          red[0][tid >> 5] = sn;
          red[1][tid >> 5] = sd;
        }
        __syncthreads();
        if (tid == 0) {
          double tn = 0.0, td = 0.0;
          for (int w = 0; w < kFcThreads / 32; ++w) {
            tn += red[0][w];
            td += red[1][w];
          }
          double* o = a.rpart + ((int64_t)fc * gridDim.x + blockIdx.x) * 2;
          o[0] = tn;
          o[1] = td;
        }
      }
      __syncthreads();
      FC_TICK(4);
    }
    const int ntask = ph ? N1 * kFcCols : 2 * N1 * kFcCols;
#pragma unroll 1
    for (int task = tid; task < ntask; task += kFcThreads) {
      const int fr = task / (N1 * kFcCols), r = task % (N1 * kFcCols);
      const int n1 = r / kFcCols, col = r % kFcCols;
      cf* b = buf0 + (fr ? B1 : 0) + col;
      cf* q[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) q[c] = b + (n1 ^ c) * S;
      cf x[N2];
#pragma unroll
      for (int m = 0; m < N2; ++m) {
        const cf v = q[m & 3][N1 * m * S];
        x[m] = ph ? conj(v) : v;
      }
      reg_dft<false, N2>(x);
      if (ph == 0) {
        const cf* tw = a.tw1 + n1;                    // w_Ph^(n1 m) at [m][n1]
#pragma unroll
        for (int m = 0; m < N2; ++m) {
          cf y = x[reg_pos<N2>(m)];
          if (m) y = y * ldg_cf(tw + N1 * m);
          q[m & 3][N1 * m * S] = y;
        }
      } else if (col < nv) {
        cf* dst = a.ihat + ((int64_t)fc * a.H + n1) * a.Pw2p + v0 + col;
        const int64_t step = (int64_t)N1 * a.Pw2p;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
          if (n1 + N1 * n2 < a.H && CBP_CHECK(v0 + col < a.Pw2p, 4)) dst[n2 * step] = conj(x[reg_pos<N2>(n2)]);
        }
      }
    }
  }
#ifdef CBP_PHASE_TIMING
  __syncthreads();
  FC_TICK(5);
  if (tid == 0 && blockIdx.x % 61 == 0 && blockIdx.y % 23 == 0)
    printf("colpass blk=%d,%d | rt %lld wait %lld step1 %lld step2 %lld step3 %lld\n", blockIdx.x,
           blockIdx.y, tck[1] - tck[0], tck[2] - tck[1], tck[3] - tck[2], tck[4] - tck[3],
           tck[5] - tck[4]);
#endif
  static_assert(N1 <= kFcMaxT, "kernel rows beyond the row-transform table");
  static_assert(N1 % 4 == 0, "the swizzle permutes rows within groups of four");
  static_assert(Ph == N1 * N2, "");
}

template <int N1, int N2, bool RESID>
void run_fused(const Plan& p, char* ws, cudaStream_t st) {
  FusedColArgs a;
  a.spec[0] = (const cf*)(ws + p.off_spec[0]);
  a.spec[1] = (const cf*)(ws + p.off_spec[1]);
  a.ihat = (cf*)(ws + p.off_ihat);
  a.krow = (const cf*)(ws + p.off_krow);
  a.tw1 = (const cf*)(ws + p.off_tw2c);
  a.tw2 = a.tw1 + N1 * N2;
  a.accepted = (!RESID && p.learned) ? (const int*)(ws + p.off_acc) : nullptr;
  a.rpart = RESID ? (double*)(ws + p.off_rpart) : nullptr;
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
  const int tm = std::max(p.t1, p.t2);
  k_kernel_rows<<<dim3((p.Pw2p + kKrThreads - 1) / kKrThreads, tm, p.n * 2), kKrThreads, 0, st>>>(
      (const double*)(ws + p.off_kd), (const cf*)(ws + p.off_tw_w), (cf*)(ws + p.off_krow), p.t1,
      p.t2, p.Pw, p.Pw2, p.Pw2p);
  const size_t sm = FcSmem<N1, N2>::kBytes;
  auto kern = k_col_deconv_fused<N1, N2, RESID>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  kern<<<dim3(fused_strips(p), p.n * p.C), kFcThreads, sm, st>>>(a);
}

}  // namespace

bool col_pass_fused(const Plan& p) {
  if (p.fft_f64 || p.single_kernel) return false;
  if (p.t1 > kFcMaxT || p.t2 > kFcMaxT) return false;
  return p.Ph == 1120 && p.Pw2p % 4 == 0;
}

int fused_strips(const Plan& p) { return (p.Pw2 + kFcCols - 1) / kFcCols; }

void launch_col_deconv_fused(const Plan& p, char* ws, cudaStream_t st) {
  run_fused<32, 35, false>(p, ws, st);
}

void launch_col_gate_fused(const Plan& p, char* ws, cudaStream_t st) {
  run_fused<32, 35, true>(p, ws, st);
  launch_gate(p, ws, st, fused_strips(p));
}

}  // namespace cbp
