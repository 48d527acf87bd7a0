// A6: dual-kernel Fourier deconvolution on a 7-smooth Ph x Pw grid.
//
//   I^ = (conj(K1^) B1^ + conj(K2^) B2^) / (|K1^|^2 + |K2^|^2 + eps),
//   latent = real(IDFT(I^))[0:H, 0:W]
//
// Section 4 recovers the latent by dividing B1 by K1 in the Fourier domain and
// Section 5 uses a vendor FFT for it; here both kernels are used (the single
// kernel form is kept as an option) and the FFTs are this file's own
// mixed-radix (2, 3, 4, 5, 7) Stockham transforms in shared memory, so any
// 7-smooth grid works.  Three passes over HBM:
//   1. row pass:     each row of B1 and B2 -> real-to-complex FFT (a
//                    half-length complex FFT when Pw is even), Pw/2+1 bins;
//   2. column pass:  per strip of spectrum columns, column FFTs of both
//                    frames, the dual-kernel formula with the kernels' spectra,
//                    inverse column FFT, rows 0..H-1 kept;
//   3. inverse rows: complex-to-real inverse FFT, crop to W, scale 1/(Ph Pw).
// Zero padding is implicit: rows >= H_Bk and columns >= W_Bk are never read.
#include "cbp_common.cuh"
#include "cbp_dft.cuh"
#include "cbp_internal.h"
#ifdef CBP_PHASE_TIMING
#include <cstdio>
#endif

namespace cbp {

CBP_CHECKS_TU(kChkFft)

// Checked builds only: bytes every bulk-copy barrier expects beyond its copies.
// Nonzero (cbp_check_expire_waits), every copy still lands but no barrier
// phase completes, so each bounded wait runs out with nothing in flight: the
// timeout path, exercised without a fault.
#ifdef CBP_CHECKS
static __device__ uint32_t cbp_tx_extra;
#define CBP_TX_EXTRA cbp_tx_extra
#else
#define CBP_TX_EXTRA 0u
#endif

namespace {

constexpr int kFftThreads = 256;

// One Stockham stage of radix R over nb transforms of length N (stride N),
// in -> out; tw = this stage's twiddles (shared memory).
template <typename T, bool Inv, int R>
__device__ __forceinline__ void stockham_stage(const cpx<T>* __restrict__ in,
                                               cpx<T>* __restrict__ out, const FftStage& st,
                                               int N, int nb, const cpx<T>* tw) {
  const int Nr = st.Nr, Ns = st.Ns;
  for (int idx = threadIdx.x; idx < nb * Nr; idx += blockDim.x) {
    const int b = st.mNr ? (int)__umulhi((unsigned)idx, st.mNr) : idx;   // idx / Nr
    const int j = idx - b * Nr;
    const int q = st.mNs ? (int)__umulhi((unsigned)j, st.mNs) : j;      // j / Ns
    const int k = j - q * Ns;
    const cpx<T>* src = in + b * N + j;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[r * Nr];
    if (Ns > 1) {
      const cpx<T>* w = tw + k;       // r-major: consecutive k are consecutive words
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cpx<T> ww = w[(r - 1) * Ns];
        if (Inv) ww.im = -ww.im;
        v[r] = v[r] * ww;
      }
    }
    small_dft<T, Inv, R>(v);
    cpx<T>* dst = out + b * N + q * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * Ns] = v[r];
  }
}

// nb transforms in shared memory (a, scratch b); returns the buffer with the
// result.  tw: the plan's stage twiddles in shared memory.  Block-wide.
template <typename T, bool Inv>
__device__ cpx<T>* fft_block(cpx<T>* a, cpx<T>* b, const FftPlan& pl, int nb, const cpx<T>* tw,
                             int first = 0) {
  for (int s = first; s < pl.nst; ++s) {
    const FftStage& st = pl.st[s];
    const cpx<T>* t = tw + st.tw;
    switch (st.R) {
      case 2: stockham_stage<T, Inv, 2>(a, b, st, pl.n, nb, t); break;
      case 3: stockham_stage<T, Inv, 3>(a, b, st, pl.n, nb, t); break;
      case 4: stockham_stage<T, Inv, 4>(a, b, st, pl.n, nb, t); break;
      case 5: stockham_stage<T, Inv, 5>(a, b, st, pl.n, nb, t); break;
      case 7: stockham_stage<T, Inv, 7>(a, b, st, pl.n, nb, t); break;
      case 8: stockham_stage<T, Inv, 8>(a, b, st, pl.n, nb, t); break;
      default: stockham_stage<T, Inv, 9>(a, b, st, pl.n, nb, t); break;
    }
    __syncthreads();
    cpx<T>* tmp = a;
    a = b;
    b = tmp;
  }
  return a;
}

// Stage twiddles of a plan: entry st.tw + (r-1) Ns + k = exp(-2 pi i k r / (Ns R)),
// r-major so that the threads of a stage (consecutive k) read consecutive entries.
// One Stockham stage with the plan fixed at compile time (radix R, stride NS,
// length N, twiddle offset TWO): strides and divisors are immediates.
template <typename T, bool Inv, int R, int NS, int N, int TWO>
__device__ __forceinline__ void stockham_stage_fixed(const cpx<T>* __restrict__ in,
                                                     cpx<T>* __restrict__ out, int nb,
                                                     const cpx<T>* tw) {
  constexpr int NR = N / R;
  for (int idx = threadIdx.x; idx < nb * NR; idx += blockDim.x) {
    const int b = idx / NR, j = idx - b * NR;
    const int q = j / NS, k = j - q * NS;
    const cpx<T>* src = in + b * N + j;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[r * NR];
    if (NS > 1) {
      const cpx<T>* w = tw + TWO + k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cpx<T> ww = w[(r - 1) * NS];
        if (Inv) ww.im = -ww.im;
        v[r] = v[r] * ww;
      }
    }
    small_dft<T, Inv, R>(v);
    cpx<T>* dst = out + b * N + q * NS * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * NS] = v[r];
  }
}

// Stages 1-3 of the fixed four-stage plan R0..R3 of N (stage 0 is fused into
// the callers' first stage); returns the buffer with the result.
template <typename T, bool Inv, int N, int R0, int R1, int R2, int R3>
__device__ __forceinline__ cpx<T>* fft_rest_fixed(cpx<T>* a, cpx<T>* b, int nb, const cpx<T>* tw) {
  constexpr int N1 = R0, N2 = R0 * R1, N3 = R0 * R1 * R2;
  constexpr int O1 = (R0 - 1), O2 = O1 + N1 * (R1 - 1), O3 = O2 + N2 * (R2 - 1);
  stockham_stage_fixed<T, Inv, R1, N1, N, O1>(a, b, nb, tw);
  __syncthreads();
  stockham_stage_fixed<T, Inv, R2, N2, N, O2>(b, a, nb, tw);
  __syncthreads();
  stockham_stage_fixed<T, Inv, R3, N3, N, O3>(a, b, nb, tw);
  __syncthreads();
  return b;
}

template <int N, int R0, int R1, int R2, int R3>
__host__ __device__ inline bool plan_is(const FftPlan& pl) {
  return pl.n == N && pl.nst == 4 && pl.st[0].R == R0 && pl.st[1].R == R1 && pl.st[2].R == R2 &&
         pl.st[3].R == R3;
}

// The row transforms' plan of the 1080p grid: half-length 972 = 9 9 4 3.
#define CBP_ROW_PLAN 972, 9, 9, 4, 3

template <typename T>
__global__ void k_stage_twiddles(FftPlan pl, cpx<T>* out) {
  for (int s = 0; s < pl.nst; ++s) {
    const FftStage& st = pl.st[s];
    const int cnt = st.Ns * (st.R - 1);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
      const int r = e / st.Ns + 1, k = e % st.Ns;
      double sn, cs;
      sincospi(-2.0 * (double)(k * r) / (double)(st.Ns * st.R), &sn, &cs);
      out[st.tw + e] = mk<T>((T)cs, (T)sn);
    }
  }
}

template <typename T>
__device__ __forceinline__ void load_twiddles(cpx<T>* dst, const cpx<T>* src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

template <typename T>
__global__ void k_twiddles(cpx<T>* tw, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)n, &s, &c);
    tw[k] = mk<T>((T)c, (T)s);
  }
}

// Kernel spectra K^_k[u][v], u < Ph, v < Pw2, from the double kernels:
// Spectra of both kernels on the Ph x Pw grid (Pw/2 + 1 columns kept):
//   K^(u, v) = sum_p w_H^(u p) R_p(v),   R_p(v) = sum_q K[p][q] w_W^(q v).
// A block takes 64 columns of one kernel: first the t row transforms R_p(v),
// then every u with each lane on two columns (v, v + 32: coalesced 256-byte
// row segments per warp store), kSpecRows rows at a time so that each R_p(v)
// read serves kSpecRows outputs; the sum over p by Horner's rule in
// z = w_H^u (one complex multiply-add per term, no twiddle indexing).
constexpr int kSpecCols = 64;
constexpr int kSpecRows = 8;

template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_kernel_spectra(const double* kd, int t1, int t2, int Ph, int Pw, int Pw2, int Pw2p,
                 const cpx<T>* tw_h, const cpx<T>* tw_w, cpx<T>* khat) {
  extern __shared__ __align__(16) char smem[];
  cpx<T>* kv = (cpx<T>*)smem;                       // [t][kSpecCols]
  cpx<T>* twh = kv + kMaxN * kSpecCols;             // [Ph]
  const int k = blockIdx.y, f = blockIdx.z;
  const int t = k ? t2 : t1;
  const double* K = kd + (int64_t)f * (t1 * t1 + t2 * t2) + (k ? t1 * t1 : 0);
  const int v0 = blockIdx.x * kSpecCols;
  for (int i = threadIdx.x; i < Ph; i += blockDim.x) twh[i] = tw_h[i];
  for (int idx = threadIdx.x; idx < t * kSpecCols; idx += blockDim.x) {
    const int p = idx / kSpecCols, vl = idx % kSpecCols, v = v0 + vl;
    cpx<T> acc = mk<T>(0, 0);
    if (v < Pw2) {
      int e = 0;                              // (v q) mod Pw, incrementally
      for (int q = 0; q < t; ++q) {
        acc = acc + (T)K[p * t + q] * tw_w[e];
        e += v;
        if (e >= Pw) e -= Pw;
      }
    }
    kv[idx] = acc;
  }
  __syncthreads();
  cpx<T>* out = khat + ((int64_t)f * 2 + k) * Ph * Pw2p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int va = v0 + lane, vb = v0 + 32 + lane;
  // Horner's rule in z = w_H^u: K^(u, v) = (...(R_{t-1}(v) z + R_{t-2}(v)) z + ...) + R_0(v)
  for (int u0 = warp * kSpecRows; u0 < Ph; u0 += nw * kSpecRows) {
    cpx<T> acc[kSpecRows][2], z[kSpecRows];
    const cpx<T> ra = kv[(t - 1) * kSpecCols + lane], rb = kv[(t - 1) * kSpecCols + 32 + lane];
#pragma unroll
    for (int j = 0; j < kSpecRows; ++j) {
      z[j] = twh[u0 + j < Ph ? u0 + j : 0];   // rows past Ph are computed as u = 0, not stored
      acc[j][0] = ra;
      acc[j][1] = rb;
    }
    for (int p = t - 2; p >= 0; --p) {
      const cpx<T> ca = kv[p * kSpecCols + lane], cb = kv[p * kSpecCols + 32 + lane];
#pragma unroll
      for (int j = 0; j < kSpecRows; ++j) {
        acc[j][0] = acc[j][0] * z[j] + ca;
        acc[j][1] = acc[j][1] * z[j] + cb;
      }
    }
#pragma unroll
    for (int j = 0; j < kSpecRows; ++j) {
      if (u0 + j < Ph) {
        cpx<T>* o = out + (int64_t)(u0 + j) * Pw2p;
        if (va < Pw2) o[va] = acc[j][0];
        if (vb < Pw2) o[vb] = acc[j][1];
      }
    }
  }
}

// ------------------------------------------------- asynchronous copies ---
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(src_bytes)
               : "memory");
}
template <int B>
__device__ __forceinline__ void cp_async_small(void* smem_dst, const void* gsrc) {   // B = 4 or 8
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bulk (TMA) copies completed on an mbarrier.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  bytes += CBP_TX_EXTRA;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// global -> this block's shared memory, `bytes` a multiple of 16, both ends 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Wait for phase `parity` of the barrier, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  const uint32_t a = smem_addr(bar);
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
constexpr int kWaitLimit = 1 << 20;

__device__ __forceinline__ cf ldg_cpx(const cf* p) {
  const float2 v = __ldg((const float2*)p);
  return mk(v.x, v.y);
}
__device__ __forceinline__ cd ldg_cpx(const cd* p) {
  const double2 v = __ldg((const double2*)p);
  return mk(v.x, v.y);
}

// ------------------------------------------ row pass (A1 folds + A6 rows) ---
//
// One read of every row of B1 and B2 serves both the evaluation folds of A1
// and the forward row FFTs of A6.  A block owns the rows r = x, x + X, x + 2X,
// ... (x = blockIdx.x, X = gridDim.x) of one frame channel; with X = M every
// row of a block has the same residue r mod M, so the block alone completes
// column-fold bin x:  Fz1[x][c] = sum_{r = x mod M} B[r][c].  Each row's own
// fold Fz2[m][r] = sum_{c = m mod M} B[r][c] is finished as the row passes.
// The bins of float32 frames are exact float sums kept as the TwoSum pair
// (hi, lo) of floats, those of float64 frames doubles (8 bytes either way);
// the M-point DFT over the bins (k_fold_dft, cbp_eval.cu) gives the samples.
//
// Rows arrive by cp.async into a double-buffered staging area, nbr rows per
// group, the next group in flight while the current one is folded and
// transformed.
struct RowPassArgs {
  const cf* tw2;       // in-register row pass: w_N^(n1 k2) at [k2][n1]
  FrameDesc fr[2];
  void* spec[2];       // cpx<T> [n][C][H_Bk][Pw2p] (FFT)
  void* bins_r[2];     // [n C][M][H_Bk] row-fold bins, 8 bytes each (FOLD)
  void* bins_c[2];     // [n C][M][W_Bk] column-fold bins (FOLD)
  int* bad;            // [n] non-finite input flags (FOLD)
  int* err;            // set when a copy does not complete in time
  int M;
  int fft_frames;      // frames whose rows are transformed (1: single-kernel form)
  int Pw, Pw2, Pw2p, half, nbr, rw;
  int wl;              // width the shared-memory layout is sized for (max W_Bk)
  FftPlan pl;          // plan of Pw/2 (half) or Pw
};

constexpr int kRowPassThreads = 512;

// Optional per-phase cycle counts of the row pass (build with
// -DCBP_PHASE_TIMING): thread 0 accumulates clock64 deltas between the phases
// and one block prints them.
#ifdef CBP_PHASE_TIMING
#define RP_MARK(i)                                  \
  do {                                              \
    if (threadIdx.x == 0) {                         \
      const long long now = clock64();              \
      rp_t[i] += now - rp_last;                     \
      rp_last = now;                                \
    }                                               \
  } while (0)
#else
#define RP_MARK(i) \
  do {             \
  } while (0)
#endif
constexpr int kRowWarps = kRowPassThreads / 32;
constexpr int kColRegs = 4;          // column-fold accumulators per thread held in registers
constexpr int kMaxRowGroup = 8;      // rows per group at most

template <typename In> struct FoldAcc;
template <> struct FoldAcc<float> { using type = TwoSum; };
template <> struct FoldAcc<double> { using type = DoubleSum; };

// Shared-memory layout of the row pass (byte offsets); one definition for the
// kernel and its launcher.  The FFT's second buffer reuses the group's staging
// rows once they are consumed, when they are large enough (b1_alias); column
// accumulators live in registers unless W exceeds kColRegs per thread.
struct RowPassSmem {
  size_t tw, b0, b1, raw0, raw1, colacc, rb, rph, mbar, total;
  bool b1_alias, col_smem;
};
__host__ __device__ inline size_t rp_align(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline RowPassSmem row_pass_layout(int N, int ntw, int W, int nbr, int rw,
                                                       size_t ce, size_t es, bool fold, bool fft) {
  RowPassSmem L;
  L.b1_alias = (size_t)N * ce <= (size_t)rw * es;
  L.col_smem = fold && W > kColRegs * kRowPassThreads;
  size_t o = 0;
  L.tw = o;
  if (fft) o += rp_align((size_t)((ntw + 1) & ~1) * ce);
  L.b0 = o;
  if (fft) o += rp_align((size_t)nbr * N * ce);
  L.b1 = o;
  if (fft && !L.b1_alias) o += rp_align((size_t)nbr * N * ce);
  L.raw0 = o;
  o += rp_align((size_t)nbr * rw * es);
  L.raw1 = o;
  o += rp_align((size_t)nbr * rw * es);
  L.colacc = o;
  if (L.col_smem) o += rp_align((size_t)W * 8);
  L.rb = o;
  if (fold) o += rp_align((size_t)kRowWarps * 32 * 8);
  L.rph = o;
  o += rp_align(2 * (size_t)nbr * sizeof(int));
  L.mbar = o;
  o += rp_align(2 * sizeof(uint64_t));
  L.total = o;
  return L;
}

// One element a thread fetched for a staging row, stored later.
template <typename In> struct Edge {
  In v;
  int at;   // index in the staging buffer, -1: none
};

// First Stockham stage (Ns = 1) of the forward row transforms, reading the
// staged float/double rows directly: element m of row i is (x[2m], x[2m+1])
// for the half-length transform (Pw even), else (x[m], 0), zero past W.
// Pairs are read as one 8-byte load when the row's phase keeps them aligned.
// NC > 0: the transform length fixed at compile time (strides and divisors
// become immediates).
template <typename T, int R, typename In, int NC = 0>
__device__ __forceinline__ void stage_first_raw(const In* raw, const int* ph, int rw, int W, bool half,
                                                cpx<T>* out, const FftStage& st, int N_, int nb) {
  const int Nr = NC ? NC / R : st.Nr, N = NC ? NC : N_;
  for (int idx = threadIdx.x; idx < nb * Nr; idx += blockDim.x) {
    const int b = NC ? idx / (NC / R) : st.mNr ? (int)__umulhi((unsigned)idx, st.mNr) : idx;
    const int j = idx - b * Nr;
    const In* row = raw + b * rw + ph[b];
    const bool pair8 = half && sizeof(In) == 4 && (ph[b] & 1) == 0;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = j + r * Nr;
      if (half) {
        const int c0 = 2 * m;
        if (pair8 && c0 + 1 < W) {
          const float2 x = *(const float2*)(row + c0);
          v[r] = mk<T>((T)x.x, (T)x.y);
        } else {
          v[r] = mk<T>(c0 < W ? (T)row[c0] : (T)0, c0 + 1 < W ? (T)row[c0 + 1] : (T)0);
        }
      } else {
        v[r] = mk<T>(m < W ? (T)row[m] : (T)0, (T)0);
      }
    }
    small_dft<T, false, R>(v);
    cpx<T>* dst = out + b * N + j * R;   // Ns = 1: outputs of butterfly j are contiguous
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r] = v[r];
  }
}

template <typename T, typename In>
__device__ __forceinline__ void first_stage_raw(const In* raw, const int* ph, int rw, int W, bool half,
                                                cpx<T>* out, const FftPlan& pl, int nb) {
  const FftStage& st = pl.st[0];
  switch (st.R) {
    case 2: stage_first_raw<T, 2, In>(raw, ph, rw, W, half, out, st, pl.n, nb); break;
    case 3: stage_first_raw<T, 3, In>(raw, ph, rw, W, half, out, st, pl.n, nb); break;
    case 4: stage_first_raw<T, 4, In>(raw, ph, rw, W, half, out, st, pl.n, nb); break;
    case 5: stage_first_raw<T, 5, In>(raw, ph, rw, W, half, out, st, pl.n, nb); break;
    case 7: stage_first_raw<T, 7, In>(raw, ph, rw, W, half, out, st, pl.n, nb); break;
    case 8: stage_first_raw<T, 8, In>(raw, ph, rw, W, half, out, st, pl.n, nb); break;
    default: stage_first_raw<T, 9, In>(raw, ph, rw, W, half, out, st, pl.n, nb); break;
  }
}

// Stage nr rows (row i at element offset rowoff(i) of fb) into the rows
// dst + i * rw, each at its own 16-byte phase ph_i (element c of row i lands at
// dst[i * rw + ph_i + c]).  Thread 0 moves each row's 16-byte-aligned body
// with one bulk (TMA) copy completing on `bar`; the few elements before the
// first and after the last 16-byte boundary are loaded by other threads into
// the returned Edge, which the caller stores before the rows are read (so the
// load's latency overlaps other work).  Nothing outside the rows is read.
template <typename In, class RowOff>
__device__ __forceinline__ Edge<In> stage_rows_bulk(In* dst, int* rph, const In* fb,
                                                    const RowOff& rowoff, int nr, int W, int rw,
                                                    uint64_t* bar) {
  constexpr int E = 16 / (int)sizeof(In);
  auto geom = [&](int i, const In*& row, int& ph, int& head, int& body) {
    row = fb + rowoff(i);
    ph = (int)(((uintptr_t)row / sizeof(In)) & (E - 1));
    head = ph ? min(E - ph, W) : 0;
    body = ((W - head) / E) * E;                    // elements in whole 16-byte chunks
  };
  if (threadIdx.x == 0) {
    uint32_t total = 0;
    for (int i = 0; i < nr; ++i) {
      const In* row;
      int ph, head, body;
      geom(i, row, ph, head, body);
      total += (uint32_t)(body * sizeof(In));
      rph[i] = ph;
    }
    mbar_expect_tx(bar, total);
    for (int i = 0; i < nr; ++i) {
      const In* row;
      int ph, head, body;
      geom(i, row, ph, head, body);
      if (body) bulk_g2s(dst + i * rw + ph + head, row + head, (uint32_t)(body * sizeof(In)), bar);
    }
  }
  Edge<In> e{(In)0, -1};
  const int t = (int)threadIdx.x - 32;   // warps other than thread 0's
  if (t >= 0 && t < nr * 2 * E) {
    const int i = t / (2 * E), sl = t - i * (2 * E);
    const In* row;
    int ph, head, body;
    geom(i, row, ph, head, body);
    const int c = sl < E ? sl : head + body + (sl - E);
    if ((sl < E && sl < head) || (sl >= E && c < W)) {
      e.v = row[c];
      e.at = i * rw + ph + c;
    }
  }
  return e;
}

template <typename T, typename In, bool FOLD, bool FFT>
__global__ void __launch_bounds__(kRowPassThreads)
k_row_pass(RowPassArgs a, const cpx<T>* tw_w, const cpx<T>* stw) {
  using Acc = typename FoldAcc<In>::type;
  extern __shared__ __align__(16) char smem[];
  const FrameDesc& fr = a.fr[blockIdx.z];
  const int N = a.pl.n, NB = a.nbr, W = fr.w, M = a.M;
  const bool fft = FFT && (int)blockIdx.z < a.fft_frames;
  const RowPassSmem L = row_pass_layout(N, a.pl.ntw, a.wl, NB, a.rw, sizeof(cpx<T>), sizeof(In),
                                        FOLD, FFT);
  cpx<T>* tw = (cpx<T>*)(smem + L.tw);
  cpx<T>* b0 = (cpx<T>*)(smem + L.b0);
  In* const raw0 = (In*)(smem + L.raw0);
  In* const raw1 = (In*)(smem + L.raw1);
  Acc* colacc = (Acc*)(smem + L.colacc);
  Acc* rb = (Acc*)(smem + L.rb);
  int* rph = (int*)(smem + L.rph);
  uint64_t* bars = (uint64_t*)(smem + L.mbar);   // one per staging buffer
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t par = 0u;   // bit b: phase parity of buffer b's next completion
  if (fft) load_twiddles(tw, stw, a.pl.ntw);
  Acc creg[kColRegs];
  if (FOLD && L.col_smem)
    for (int c = threadIdx.x; c < W; c += blockDim.x) colacc[c] = Acc();
  const int fc = blockIdx.y, f = fc / fr.c, ch = fc % fr.c;
  const int x0 = blockIdx.x, X = gridDim.x;
  const int nrows = x0 < fr.h ? (fr.h - x0 + X - 1) / X : 0;
  const int ngroups = (nrows + NB - 1) / NB;
  const In* fb = (const In*)frame_base(fr, f) + (int64_t)ch * fr.cs;
  auto row_of = [&](int g, int i) { return x0 + (g * NB + i) * X; };
  if (ngroups > 0) {
    const Edge<In> e0 = stage_rows_bulk<In>(raw0, rph, fb,
                                            [&](int i) { return (int64_t)row_of(0, i) * fr.rs; },
                                            min(NB, nrows), W, a.rw, &bars[0]);
    if (e0.at >= 0) raw0[e0.at] = e0.v;
  }
  cpx<T>* spec = fft ? (cpx<T>*)a.spec[blockIdx.z] + (int64_t)fc * fr.h * a.Pw2p : nullptr;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#ifdef CBP_PHASE_TIMING
  long long rp_t[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long rp_last = clock64();
#endif
  for (int g = 0; g < ngroups; ++g) {
    const int nr = min(NB, nrows - g * NB);
    RP_MARK(7);
    Edge<In> en{(In)0, -1};
    if (g + 1 < ngroups) {
      const int g1 = g + 1;
      en = stage_rows_bulk<In>((g1 & 1) ? raw1 : raw0, rph + (g1 & 1) * NB, fb,
                               [&](int i) { return (int64_t)row_of(g1, i) * fr.rs; },
                               min(NB, nrows - g1 * NB), W, a.rw, &bars[g1 & 1]);
    }
    RP_MARK(0);
    const bool arrived = mbar_wait(&bars[g & 1], (par >> (g & 1)) & 1u, kWaitLimit);
    par ^= 1u << (g & 1);
    if (__syncthreads_or(!arrived)) {
      // a copy did not complete in time: report it, wait (bounded) for the
      // other buffer's copies still in flight, and leave
      if (threadIdx.x == 0) atomicOr(a.err, 1);
      if (g + 1 < ngroups) mbar_wait(&bars[(g + 1) & 1], (par >> ((g + 1) & 1)) & 1u, kWaitLimit);
      return;
    }
    RP_MARK(1);
    In* const rw0 = (g & 1) ? raw1 : raw0;
    const int* ph = rph + (g & 1) * NB;
    if (FOLD) {
      // element c of staged row i is rw0[roff(i) + c]
      auto roff = [&](int i) { return i * a.rw + ph[i]; };
      // column folds: this block's bin, one thread per column (full groups
      // without per-row tests)
      if (!L.col_smem) {
        if (nr == kMaxRowGroup) {
          int off[kMaxRowGroup];
#pragma unroll
          for (int i = 0; i < kMaxRowGroup; ++i) off[i] = roff(i);
#pragma unroll
          for (int j = 0; j < kColRegs; ++j) {
            const int c = threadIdx.x + j * kRowPassThreads;
            if (c < W) {
#pragma unroll
              for (int i = 0; i < kMaxRowGroup; ++i) creg[j].add(rw0[off[i] + c]);
            }
          }
        } else {
          for (int i = 0; i < nr; ++i) {
            const In* rp = rw0 + roff(i);
#pragma unroll
            for (int j = 0; j < kColRegs; ++j) {
              const int c = threadIdx.x + j * kRowPassThreads;
              if (c < W) creg[j].add(rp[c]);
            }
          }
        }
      } else {
        for (int c = threadIdx.x; c < W; c += blockDim.x) {
          Acc acc = colacc[c];
          for (int i = 0; i < nr; ++i) acc.add(rw0[roff(i) + c]);
          colacc[c] = acc;
        }
      }
      // row folds: task (i, sg, m) sums columns c = m mod M of row i over
      // segment sg; nseg segments per (row, bin) fill the block.  Only the
      // last step of a row can pass W; two accumulators for latency.
      const int nseg = max(1, kRowPassThreads / (nr * M));
      const int nsteps = (W + M - 1) / M, sps = (nsteps + nseg - 1) / nseg;
      const int t = threadIdx.x;
      if (t < nr * M * nseg) {
        const int i = t / (M * nseg), r = t - i * (M * nseg), sg = r / M, m = r - sg * M;
        Acc acc, acc2;
        const In* rp = rw0 + roff(i);
        const int st0 = sg * sps, e = min(nsteps, st0 + sps), ef = min(e, nsteps - 1);
        int st = st0, c = st0 * M + m;
        for (; st + 1 < ef; st += 2, c += 2 * M) {
          acc.add(rp[c]);
          acc2.add(rp[c + M]);
        }
        if (st < ef) {
          acc.add(rp[c]);
          ++st;
          c += M;
        }
        if (st < e && c < W) acc.add(rp[c]);
        acc.merge(acc2);
        rb[t] = acc;
      }
    }
    RP_MARK(2);
    // first FFT stage straight from the staging rows into b0
    if (fft) {
      if (plan_is<CBP_ROW_PLAN>(a.pl))
        stage_first_raw<T, 9, In, 972>(rw0, ph, a.rw, W, a.half, b0, a.pl.st[0], 972, nr);
      else
        first_stage_raw<T, In>(rw0, ph, a.rw, W, a.half, b0, a.pl, nr);
    }
    __syncthreads();
    RP_MARK(3);
    if (FOLD) {
      const int nseg = max(1, kRowPassThreads / (nr * M));
      for (int t = threadIdx.x; t < nr * M; t += blockDim.x) {
        const int i = t / M, m = t - i * M;
        Acc v = rb[(i * nseg) * M + m];
        for (int sg = 1; sg < nseg; ++sg) v.merge(rb[(i * nseg + sg) * M + m]);
        v.store((char*)a.bins_r[blockIdx.z] + 8 * (((int64_t)fc * M + m) * fr.h + row_of(g, i)));
      }
    }
    if (fft) {
      // the staging rows of this group are consumed: they serve as the
      // FFT's second buffer when large enough
      cpx<T>* b1 = L.b1_alias ? (cpx<T>*)rw0 : (cpx<T>*)(smem + L.b1);
      cpx<T>* Z = plan_is<CBP_ROW_PLAN>(a.pl) ? fft_rest_fixed<T, false, CBP_ROW_PLAN>(b0, b1, nr, tw)
                                              : fft_block<T, false>(b0, b1, a.pl, nr, tw, 1);
      RP_MARK(4);
      // a thread keeps its output columns k (and their twiddle) over the rows
      for (int k = threadIdx.x; k < a.Pw2; k += blockDim.x) {
        if (a.half) {
          const int ka = k < N ? k : 0, kb = k > 0 ? N - k : 0;
          const cpx<T> w = tw_w[k];                 // X = e - i w d, w = exp(-2 pi i k / Pw)
          for (int i = 0; i < nr; ++i) {
            const cpx<T>* z = Z + i * N;
            const cpx<T> zk = z[ka], zc = conj(z[kb]);
            const cpx<T> e = (T)0.5 * (zk + zc), d = (T)0.5 * (zk - zc);
            const cpx<T> wd = w * d;
            spec[(int64_t)row_of(g, i) * a.Pw2p + k] = mk<T>(e.re + wd.im, e.im - wd.re);
          }
        } else {
          for (int i = 0; i < nr; ++i) spec[(int64_t)row_of(g, i) * a.Pw2p + k] = Z[i * N + k];
        }
      }
    }
    RP_MARK(5);
    // the next group's edge elements (their buffer is not touched by this group)
    if (en.at >= 0) (((g + 1) & 1) ? raw1 : raw0)[en.at] = en.v;
    // this group's staging rows (also the FFT's scratch) are rewritten by the
    // next bulk copy: order their generic-proxy accesses before it
    fence_proxy_async();
    __syncthreads();
    RP_MARK(6);
  }
#ifdef CBP_PHASE_TIMING
  if (threadIdx.x == 0 && blockIdx.x == 1 && blockIdx.y < 2)
    printf("row_pass fold=%d fft=%d z=%d groups=%d nb=%d | issue %lld wait %lld folds %lld convert+sync %lld "
           "fft %lld post %lld endsync %lld loop %lld\n", (int)FOLD, (int)fft, (int)blockIdx.z,
           ngroups, NB, rp_t[0], rp_t[1], rp_t[2], rp_t[3], rp_t[4], rp_t[5], rp_t[6], rp_t[7]);
#endif
  if (FOLD) {
    bool finite = true;
    char* dst = (char*)a.bins_c[blockIdx.z] + 8 * (((int64_t)fc * M + x0) * W);
    if (!L.col_smem) {
#pragma unroll
      for (int j = 0; j < kColRegs; ++j) {
        const int c = threadIdx.x + j * kRowPassThreads;
        if (c < W) {
          finite = finite && creg[j].finite();
          creg[j].store(dst + 8 * (size_t)c);
        }
      }
    } else {
      for (int c = threadIdx.x; c < W; c += blockDim.x) {
        finite = finite && colacc[c].finite();
        colacc[c].store(dst + 8 * (size_t)c);
      }
    }
    if (__syncthreads_or(!finite) && threadIdx.x == 0) atomicOr(a.bad + f, 1);
  }
}

// ------------------------- row pass with in-register transforms (float rows)
//
// The same work as k_row_pass (one read of every row: A1's exact folds and
// A6's forward real row FFT) for float32 frames whose rows start on 8-byte
// boundaries and whose half-length transform N = N1 N2 splits into two
// register-sized factors (the 1080p grid: 972 = 36 x 27).  The half-length
// complex row z[m] = (x[2m], x[2m+1]) is transformed in place in the staging
// buffer by the two-factor split n = n1 + N1 n2, k = k2 + N2 k1:
//   step 1: per (row, n1), an N2-point DFT over n2 in registers, twiddled by
//           w_N^(n1 k2), back into the same slots n1 + N1 k2;
//   step 2: per (row, k2), an N1-point DFT over the slots n1 + N1 k2 in
//           registers: X[k2 + N2 k1] into slot k1 + N1 k2;
//   then the real-FFT split of X[k] and X[N - k] into the Pw/2 + 1 stored bins.
// One staging buffer of kIrRows rows: the group's rows arrive by bulk copy,
// the folds read them, the transforms overwrite them, the next group's copy is
// issued once the bins are out.  Registers, not shared memory, hold the
// transform data; two 256-thread blocks per SM.
constexpr int kIrThreads = 256;      // eight warps: two blocks keep four warps per scheduler
constexpr int kIrRows = 7;           // rows per group: 7 x 36 step-1 tasks, one warp per row in step 2

struct RowIrSmem {
  size_t tw, tw2, raw, colacc, rb, rph, mbar, total;
};
__host__ __device__ inline RowIrSmem row_ir_layout(int rw) {
  RowIrSmem L;
  size_t o = 0;
  L.tw = o;                                       // w_Pw^k, k < Pw = rw - 4
  o += rp_align((size_t)(rw - 4) * sizeof(cf));
  L.tw2 = o;                                      // step 1's w_N^(n1 k2) at [k2][n1], N = Pw / 2
  o += rp_align((size_t)(rw - 4) / 2 * sizeof(cf));
  L.raw = o;
  o += rp_align((size_t)kIrRows * rw * sizeof(float));
  L.colacc = o;                                   // column-fold (hi, lo) per column, W <= rw
  o += rp_align((size_t)rw * sizeof(TwoSum));
  L.rb = o;
  o += rp_align((size_t)kIrThreads * 8);
  L.rph = o;
  o += rp_align((size_t)kIrRows * sizeof(int));
  L.mbar = o;
  o += rp_align(sizeof(uint64_t));
  L.total = o;
  return L;
}

template <int N1, int N2, bool FOLD>
__global__ void __launch_bounds__(kIrThreads, 2)
k_row_pass_ir(RowPassArgs a, const cf* tw_w) {
  constexpr int N = N1 * N2;
  extern __shared__ __align__(16) char smem[];
  const FrameDesc& fr = a.fr[blockIdx.z];
  const int W = fr.w, M = a.M, rw = a.rw;
  const bool fft = (int)blockIdx.z < a.fft_frames;
  const RowIrSmem L = row_ir_layout(rw);
  float* const raw = (float*)(smem + L.raw);
  TwoSum* rb = (TwoSum*)(smem + L.rb);
  int* rph = (int*)(smem + L.rph);
  uint64_t* bar = (uint64_t*)(smem + L.mbar);
  cf* tws = (cf*)(smem + L.tw);
  cf* tw2s = (cf*)(smem + L.tw2);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (fft)
    for (int k = tid; k < 2 * N; k += kIrThreads) {
      tws[k] = ldg_cpx(tw_w + k);
      if (k < N) tw2s[k] = ldg_cpx(a.tw2 + k);
    }
  __syncthreads();
  uint32_t par = 0u;
  const int fc = blockIdx.y, f = fc / fr.c, ch = fc % fr.c;
  const int x0 = blockIdx.x, X = gridDim.x;
  const int nrows = x0 < fr.h ? (fr.h - x0 + X - 1) / X : 0;
  const int ngroups = (nrows + kIrRows - 1) / kIrRows;
  const float* fb = (const float*)frame_base(fr, f) + (int64_t)ch * fr.cs;
  auto row_of = [&](int g, int i) { return x0 + (g * kIrRows + i) * X; };
  cf* spec = fft ? (cf*)a.spec[blockIdx.z] + (int64_t)fc * fr.h * a.Pw2p : nullptr;
  // column folds: this thread's column pairs (c, c + 1), c = 2 (tid + kIrThreads j),
  // accumulated in shared memory across the groups
  constexpr int kColPairs = 4;
  TwoSum* colacc = (TwoSum*)(smem + L.colacc);
  if (FOLD)
    for (int c = tid; c < W; c += kIrThreads) colacc[c] = TwoSum();
  Edge<float> en{0.f, -1};
  if (ngroups > 0)
    en = stage_rows_bulk<float>(raw, rph, fb, [&](int i) { return (int64_t)row_of(0, i) * fr.rs; },
                                min(kIrRows, nrows), W, rw, bar);
  for (int g = 0; g < ngroups; ++g) {
    const int nr = min(kIrRows, nrows - g * kIrRows);
    const bool arrived = mbar_wait(bar, par, kWaitLimit);
    par ^= 1u;
    if (__syncthreads_or(!arrived)) {
      // the group's copy did not complete in time (no other copy is in flight)
      if (tid == 0) atomicOr(a.err, 1);
      return;
    }
    if (en.at >= 0) raw[en.at] = en.v;
    // zero each row past W up to the transform length (and rows past nr)
    for (int e = tid; e < nr * (2 * N - W); e += kIrThreads) {
      const int i = e / (2 * N - W), c = W + e - i * (2 * N - W);
      if (CBP_CHECK(i < kIrRows && rph[i] + c < rw, 0)) raw[i * rw + rph[i] + c] = 0.f;
    }
    __syncthreads();
    if (FOLD) {
      // column folds (this block's bin), float pairs
#pragma unroll
      for (int j = 0; j < kColPairs; ++j) {
        const int c = 2 * (tid + kIrThreads * j);
        if (c < W) {
          const float4 h = *(const float4*)(colacc + c);    // (hi, lo) of c and c + 1
          TwoSum s0, s1;
          s0.hi = h.x;
          s0.lo = h.y;
          s1.hi = h.z;
          s1.lo = h.w;
          for (int i = 0; i < nr; ++i) {
            const float2 v = *(const float2*)(raw + i * rw + rph[i] + c);
            s0.add(v.x);
            s1.add(v.y);                     // column W (odd W) reads the zeroed tail
          }
          *(float4*)(colacc + c) = make_float4(s0.hi, s0.lo, s1.hi, s1.lo);
        }
      }
      // row folds: task (i, sg, m) sums columns c = m (mod M) of row i over
      // segment sg; columns W..2N-1 read the zeroed tail
      const int nseg = max(1, kIrThreads / (nr * M));
      const int nsteps = (W + M - 1) / M, sps = (nsteps + nseg - 1) / nseg;
      if (tid < nr * M * nseg) {
        const int i = tid / (M * nseg), r = tid - i * (M * nseg), sg = r / M, m = r - sg * M;
        TwoSum acc, acc2;
        const int st0 = sg * sps, e = min(nsteps, st0 + sps);
        const float* rp = raw + i * rw + rph[i] + st0 * M + m;
        int n = e - st0;                                   // terms of this task
        const int last = st0 * M + m + (n - 1) * M;        // column of the last term
        if (n > 0 && last >= 2 * N) --n;                   // past the zeroed tail: beyond W
        int k = 0;
        for (; k + 3 < n; k += 4, rp += 4 * M) {
          acc.add(rp[0]);
          acc2.add(rp[M]);
          acc.add(rp[2 * M]);
          acc2.add(rp[3 * M]);
        }
        for (; k < n; ++k, rp += M) acc.add(rp[0]);
        acc.merge(acc2);
        rb[tid] = acc;
      }
    }
    __syncthreads();
    if (FOLD) {
      const int nseg = max(1, kIrThreads / (nr * M));
      for (int t = tid; t < nr * M; t += kIrThreads) {
        const int i = t / M, m = t - i * M;
        TwoSum v = rb[(i * nseg) * M + m];
        for (int sg = 1; sg < nseg; ++sg) v.merge(rb[(i * nseg + sg) * M + m]);
        if (CBP_CHECK(row_of(g, i) < fr.h && (i * nseg + nseg) * M <= kIrThreads, 1))
          v.store((char*)a.bins_r[blockIdx.z] + 8 * (((int64_t)fc * M + m) * fr.h + row_of(g, i)));
      }
    }
    if (fft) {
      // ---- step 1: N2-point DFTs over n2 for each (row, n1); the results go
      // to slot (n1 ^ sw(k2)) + N1 k2 of the row, sw(k2) = (k2 >> 2) & 3, so
      // that step 2's lanes (consecutive k2) fall on distinct banks.  Every
      // task reads before any writes (a barrier between).
      const bool t1 = tid < nr * N1;
      const int i1 = tid / N1, n1 = tid - i1 * N1;
      cf x1[N2];
      if (t1) {
        const cf* z = (const cf*)(raw + i1 * rw + rph[i1]) + n1;
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) x1[n2] = z[N1 * n2];
        reg_dft<false, N2>(x1);
        const cf* tw = tw2s + n1;                     // w_N^(n1 k2) at [k2][n1]: lanes read in a row
#pragma unroll
        for (int k2 = 1; k2 < N2; ++k2) x1[reg_pos<N2>(k2)] = x1[reg_pos<N2>(k2)] * tw[N1 * k2];
      }
      __syncthreads();
      if (t1) {
        cf* z = (cf*)(raw + i1 * rw + rph[i1]);
        cf* q[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] = z + (n1 ^ c);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) q[(k2 >> 2) & 3][N1 * k2] = x1[reg_pos<N2>(k2)];
      }
      __syncthreads();
      // ---- step 2: one warp per row, lane k2: an N1-point DFT over n1 gives
      // X[k2 + N2 k1] in registers; the real-FFT split pairs X[k] with
      // X[N - k], held by lane N2 - k2 at k1' = N1 - 1 - k1 (lane 0: by
      // itself at (N1 - k1) mod N1), fetched by shuffle; bins go straight out.
      const int warp = tid >> 5, lane = tid & 31;
      static_assert(N2 <= 32, "one lane per k2");
      if (warp < nr && lane < N2) {
        const int i = warp, k2 = lane;
        const cf* z = (const cf*)(raw + i * rw + rph[i]) + N1 * k2;
        const int sw = (k2 >> 2) & 3;
        const cf* q[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) q[c] = z + (c ^ sw);
        cf x[N1];
#pragma unroll
        for (int n = 0; n < N1; ++n) x[n] = q[n & 3][n & ~3];
        reg_dft<false, N1>(x);
        constexpr unsigned kMask = (N2 == 32) ? 0xffffffffu : ((1u << N2) - 1u);
        const int src = k2 ? N2 - k2 : 0;
        cf* out = spec + (int64_t)row_of(g, i) * a.Pw2p;
        (void)CBP_CHECK(N < a.Pw2p && row_of(g, i) < fr.h && rph[i] + 2 * N <= rw, 2);
        const cf* tw = tws + k2;
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          const cf send = x[reg_pos<N1>(N1 - 1 - k1)];
          const float pr = __shfl_sync(kMask, send.re, src);
          const float pi = __shfl_sync(kMask, send.im, src);
          const cf zk = x[reg_pos<N1>(k1)];
          const cf own = x[reg_pos<N1>((N1 - k1) % N1)];
          const cf zc = k2 ? mk(pr, -pi) : conj(own);
          const cf ev = 0.5f * (zk + zc), d = 0.5f * (zk - zc);
          const cf wd = tw[N2 * k1] * d;               // X = e - i w d, w = w_Pw^k
          out[k2 + N2 * k1] = mk(ev.re + wd.im, ev.im - wd.re);
        }
        if (k2 == 0) {                                 // bin N from X[0]
          const cf z0 = x[reg_pos<N1>(0)];
          const cf wd = tws[N] * mk(0.f, z0.im);       // d = i Im X[0]
          out[N] = mk(z0.re + wd.im, -wd.re);
        }
      }
    }
    // the buffer is rewritten by the next bulk copy: order its generic-proxy
    // accesses first
    fence_proxy_async();
    __syncthreads();
    if (g + 1 < ngroups) {
      const int g1 = g + 1;
      en = stage_rows_bulk<float>(raw, rph, fb, [&](int i) { return (int64_t)row_of(g1, i) * fr.rs; },
                                  min(kIrRows, nrows - g1 * kIrRows), W, rw, bar);
    }
  }
  if (FOLD) {
    bool finite = true;
    char* dst = (char*)a.bins_c[blockIdx.z] + 8 * (((int64_t)fc * M + x0) * W);
    __syncthreads();
    for (int c = tid; c < W; c += kIrThreads) {
      finite = finite && colacc[c].finite();
      colacc[c].store(dst + 8 * (size_t)c);
    }
    if (__syncthreads_or(!finite) && tid == 0) atomicOr(a.bad + f, 1);
  }
}

constexpr int kColThreads = 512;

struct ColArgs {
  void* spec[2];      // cpx<T> [n][C][H_Bk][Pw2p]
  const void* khat;   // cpx<T> [n][2][Ph][Pw2p]
  void* ihat;         // cpx<T> [n][C][H][Pw2p]
  const void* stw;    // stage twiddles of the Ph plan (read through L1)
  int H1, H2, H, C, Ph, Pw, Pw2, Pw2p, single;
  double eps;
  double* rpart;      // residual mode: [n][C][strips][2] partial sums
  FftPlan pl;         // plan of Ph
};

// Stockham stage over NB transforms interleaved in shared memory: element j
// of transform b at j * NB + b (consecutive threads take consecutive b).
template <typename T, bool Inv, int R, int NB>
__device__ __forceinline__ void stockham_stage_il(const cpx<T>* __restrict__ in,
                                                  cpx<T>* __restrict__ out, const FftStage& st,
                                                  const cpx<T>* __restrict__ tw) {
  const int Nr = st.Nr, Ns = st.Ns;
  for (int idx = threadIdx.x; idx < NB * Nr; idx += blockDim.x) {
    const int b = idx % NB, j = idx / NB;
    const int q = st.mNs ? (int)__umulhi((unsigned)j, st.mNs) : j;
    const int k = j - q * Ns;
    const cpx<T>* src = in + j * NB + b;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[r * Nr * NB];
    if (Ns > 1) {
      const cpx<T>* w = tw + st.tw + k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cpx<T> ww = ldg_cpx(w + (r - 1) * Ns);
        if (Inv) ww.im = -ww.im;
        v[r] = v[r] * ww;
      }
    }
    small_dft<T, Inv, R>(v);
    cpx<T>* dst = out + (q * Ns * R + k) * NB + b;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * Ns * NB] = v[r];
  }
}

template <typename T, bool Inv, int NB>
__device__ cpx<T>* fft_block_il(cpx<T>* a, cpx<T>* b, const FftPlan& pl, const cpx<T>* tw) {
  for (int s = 0; s < pl.nst; ++s) {
    const FftStage& st = pl.st[s];
    switch (st.R) {
      case 2: stockham_stage_il<T, Inv, 2, NB>(a, b, st, tw); break;
      case 3: stockham_stage_il<T, Inv, 3, NB>(a, b, st, tw); break;
      case 4: stockham_stage_il<T, Inv, 4, NB>(a, b, st, tw); break;
      case 5: stockham_stage_il<T, Inv, 5, NB>(a, b, st, tw); break;
      case 7: stockham_stage_il<T, Inv, 7, NB>(a, b, st, tw); break;
      case 8: stockham_stage_il<T, Inv, 8, NB>(a, b, st, tw); break;
      default: stockham_stage_il<T, Inv, 9, NB>(a, b, st, tw); break;
    }
    __syncthreads();
    cpx<T>* tmp = a;
    a = b;
    b = tmp;
  }
  return a;
}

// The same transform with the plan fixed at compile time (four stages,
// radices R0..R3 of N): every stride, twiddle offset and divisor becomes an
// immediate, so the stage's loads and stores index from one base register.
// Plans of other sizes take fft_block_il.
template <typename T, bool Inv, int R, int NS, int N, int NB, int TWO, int NT>
__device__ __forceinline__ void stockham_stage_il_fixed(const cpx<T>* __restrict__ in,
                                                        cpx<T>* __restrict__ out,
                                                        const cpx<T>* __restrict__ tw) {
  constexpr int NR = N / R;
  for (int idx = threadIdx.x; idx < NB * NR; idx += NT) {
    const int b = idx % NB, j = idx / NB;
    const int q = j / NS, k = j - q * NS;
    const cpx<T>* src = in + j * NB + b;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[r * NR * NB];
    if (NS > 1) {
      const cpx<T>* w = tw + TWO + k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cpx<T> ww = ldg_cpx(w + (r - 1) * NS);
        if (Inv) ww.im = -ww.im;
        v[r] = v[r] * ww;
      }
    }
    small_dft<T, Inv, R>(v);
    cpx<T>* dst = out + (q * NS * R + k) * NB + b;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * NS * NB] = v[r];
  }
}

// The same stage for single precision and four interleaved transforms with a
// thread on two neighbouring transforms: one 16-byte shared access per element
// pair, and the index work and twiddles of a butterfly serve both.
template <bool Inv, int R, int NS, int N, int TWO, int NT>
__device__ __forceinline__ void stockham_stage_il_fixed_x2(const cf* __restrict__ in,
                                                           cf* __restrict__ out,
                                                           const cf* __restrict__ tw) {
  constexpr int NR = N / R;
  for (int idx = threadIdx.x; idx < 2 * NR; idx += NT) {
    const int h = idx & 1, j = idx >> 1;
    const int q = j / NS, k = j - q * NS;
    const float4* src = reinterpret_cast<const float4*>(in + j * 4 + 2 * h);
    cf v0[R], v1[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 x = src[r * NR * 2];
      v0[r] = mk(x.x, x.y);
      v1[r] = mk(x.z, x.w);
    }
    if (NS > 1) {
      const cf* w = tw + TWO + k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cf ww = ldg_cpx(w + (r - 1) * NS);
        if (Inv) ww.im = -ww.im;
        v0[r] = v0[r] * ww;
        v1[r] = v1[r] * ww;
      }
    }
    small_dft<float, Inv, R>(v0);
    small_dft<float, Inv, R>(v1);
    float4* dst = reinterpret_cast<float4*>(out + (q * NS * R + k) * 4 + 2 * h);
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * NS * 2] = make_float4(v0[r].re, v0[r].im, v1[r].re, v1[r].im);
  }
}

template <typename T, bool Inv, int NB, int NT, int N, int R0, int R1, int R2, int R3>
__device__ __forceinline__ cpx<T>* fft_il_fixed(cpx<T>* a, cpx<T>* b, const cpx<T>* tw) {
  constexpr int N1 = R0, N2 = R0 * R1, N3 = R0 * R1 * R2;
  constexpr int O1 = (R0 - 1), O2 = O1 + N1 * (R1 - 1), O3 = O2 + N2 * (R2 - 1);
  if constexpr (sizeof(T) == 4 && NB == 4) {
    stockham_stage_il_fixed_x2<Inv, R0, 1, N, 0, NT>(a, b, tw);
    __syncthreads();
    stockham_stage_il_fixed_x2<Inv, R1, N1, N, O1, NT>(b, a, tw);
    __syncthreads();
    stockham_stage_il_fixed_x2<Inv, R2, N2, N, O2, NT>(a, b, tw);
    __syncthreads();
    stockham_stage_il_fixed_x2<Inv, R3, N3, N, O3, NT>(b, a, tw);
    __syncthreads();
  } else {
    stockham_stage_il_fixed<T, Inv, R0, 1, N, NB, 0, NT>(a, b, tw);
    __syncthreads();
    stockham_stage_il_fixed<T, Inv, R1, N1, N, NB, O1, NT>(b, a, tw);
    __syncthreads();
    stockham_stage_il_fixed<T, Inv, R2, N2, N, NB, O2, NT>(a, b, tw);
    __syncthreads();
    stockham_stage_il_fixed<T, Inv, R3, N3, N, NB, O3, NT>(b, a, tw);
    __syncthreads();
  }
  return a;
}

// Column transforms of the column pass: the fixed plan of the 1080p grid
// (Ph = 1120 = 7 8 5 4) or the general one.
template <typename T, bool Inv, int NB>
__device__ __forceinline__ cpx<T>* fft_il(cpx<T>* a, cpx<T>* b, const FftPlan& pl,
                                          const cpx<T>* tw) {
  if (plan_is<1120, 7, 8, 5, 4>(pl))
    return fft_il_fixed<T, Inv, NB, kColThreads, 1120, 7, 8, 5, 4>(a, b, tw);
  return fft_block_il<T, Inv, NB>(a, b, pl, tw);
}

// 1 / x: the correctly rounded single-precision reciprocal, or a double division.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Asynchronous copy of a CW-column strip of one spectrum (rows < Hk; rows
// Hk..Ph-1 and columns >= Pw2 zero-filled) into an interleaved buffer.
template <typename T, int CW>
__device__ __forceinline__ void load_strip_async(cpx<T>* dst, const cpx<T>* src, int Hk, int Ph,
                                                 int Pw2p, int ncols) {
  constexpr int E16 = 16 / (int)sizeof(cpx<T>);     // elements per 16-byte chunk
  constexpr int CH = CW / E16;                      // chunks per row
  static_assert(kColThreads % CH == 0, "column pass: threads per strip row");
  constexpr int kStep = kColThreads / CH;           // a thread keeps its chunk column
  const int c = threadIdx.x % CH;
  const int vbytes = min(E16, max(0, ncols - c * E16)) * (int)sizeof(cpx<T>);
  const cpx<T>* g = src + (int64_t)(threadIdx.x / CH) * Pw2p + c * E16;
  const int64_t gstep = (int64_t)kStep * Pw2p;
  for (int u = threadIdx.x / CH; u < Ph; u += kStep, g += gstep) {
    const int valid = u < Hk ? vbytes : 0;
    cp_async16(dst + u * CW + c * E16, valid ? g : src, valid);
  }
  cp_async_commit();
}

// Column FFTs of both spectra, dual-kernel formula, inverse column FFT.  Both
// frames' strips are fetched asynchronously up front; the second arrives
// while the first is transformed.  Three interleaved buffers of CW columns.
//
// Residual mode (RESID, learned path): instead of deconvolving, the strip's
// part of the consistency residual of the kernels in khat,
//   sum |K2^ B1^ - K1^ B2^|^2 and sum |B1^|^2  over the strip's (u, v),
// each half-spectrum column counted twice except v = 0 and v = Pw/2 (its own
// mirror); by Parseval their ratio is rho^2 of the circular convolutions.
template <typename T, int CW, bool RESID>
__global__ void __launch_bounds__(kColThreads, 2)
k_col_deconv(ColArgs a) {
  extern __shared__ __align__(16) char smem[];
  const int Ph = a.Ph;
  cpx<T>* buf0 = (cpx<T>*)smem;
  cpx<T>* buf1 = buf0 + CW * Ph;
  cpx<T>* buf2 = buf1 + CW * Ph;
  const cpx<T>* tw = (const cpx<T>*)a.stw;
  const int fc = blockIdx.y, f = fc / a.C;
  const int v0 = blockIdx.x * CW;
  const int nv = min(CW, a.Pw2 - v0);
  load_strip_async<T, CW>(buf0, (const cpx<T>*)a.spec[0] + (int64_t)fc * a.H1 * a.Pw2p + v0, a.H1,
                          Ph, a.Pw2p, nv);
  if (!a.single)
    load_strip_async<T, CW>(buf2, (const cpx<T>*)a.spec[1] + (int64_t)fc * a.H2 * a.Pw2p + v0,
                            a.H2, Ph, a.Pw2p, nv);
  if (a.single) cp_async_wait<0>();
  else cp_async_wait<1>();
  __syncthreads();
  cpx<T>* r1 = fft_il<T, false, CW>(buf0, buf1, a.pl, tw);
  cpx<T>* free1 = r1 == buf0 ? buf1 : buf0;
  cpx<T>* r2 = nullptr;
  cpx<T>* free2 = nullptr;
  if (!a.single) {
    cp_async_wait<0>();
    __syncthreads();
    r2 = fft_il<T, false, CW>(buf2, free1, a.pl, tw);
    free2 = r2 == buf2 ? free1 : buf2;
  }
  const cpx<T>* K1 = (const cpx<T>*)a.khat + ((int64_t)f * 2 + 0) * Ph * a.Pw2p + v0;
  const cpx<T>* K2 = (const cpx<T>*)a.khat + ((int64_t)f * 2 + 1) * Ph * a.Pw2p + v0;
  if (RESID) {
    // a thread keeps one column and steps down the rows; its sums (about
    // Ph / kRowStep terms) in the spectra's precision, the block's in double
    double num = 0.0, den = 0.0;
    constexpr int kRowStep = kColThreads / CW;
    const int vl = threadIdx.x % CW, v = v0 + vl;
    if (vl < nv) {
      const int64_t kstep = (int64_t)kRowStep * a.Pw2p;
      const cpx<T>* k1p = K1 + (int64_t)(threadIdx.x / CW) * a.Pw2p + vl;
      const cpx<T>* k2p = K2 + (int64_t)(threadIdx.x / CW) * a.Pw2p + vl;
      T tn = (T)0, td = (T)0;
      for (int idx = threadIdx.x; idx < CW * Ph; idx += kColThreads, k1p += kstep, k2p += kstep) {
        const cpx<T> k1 = ldg_cpx(k1p), k2 = ldg_cpx(k2p);
        const cpx<T> r = k2 * r1[idx] - k1 * r2[idx];
        tn += abs2(r);
        td += abs2(r1[idx]);
      }
      const double wv = (v == 0 || 2 * v == a.Pw) ? 1.0 : 2.0;
      num = wv * (double)tn;
      den = wv * (double)td;
    }
    __shared__ double red[2][kColThreads / 32];
    num = warp_sum(num);
    den = warp_sum(den);
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = num;
      red[1][threadIdx.x >> 5] = den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sn = 0.0, sd = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        sn += red[0][w];
        sd += red[1][w];
      }
      double* o = a.rpart + ((int64_t)fc * gridDim.x + blockIdx.x) * 2;
      o[0] = sn;
      o[1] = sd;
    }
    return;
  }
  const T eps = (T)a.eps;
  // a thread keeps one column (kColThreads is a multiple of CW) and steps
  // down the rows
  static_assert(kColThreads % CW == 0, "column pass: threads per row group");
  constexpr int kRowStep = kColThreads / CW;
  const int vl = threadIdx.x % CW;
  if (vl < nv) {
    const int64_t kstep = (int64_t)kRowStep * a.Pw2p;
    const cpx<T>* k1p = K1 + (int64_t)(threadIdx.x / CW) * a.Pw2p + vl;
    const cpx<T>* k2p = K2 + (int64_t)(threadIdx.x / CW) * a.Pw2p + vl;
    for (int idx = threadIdx.x; idx < CW * Ph; idx += kColThreads, k1p += kstep, k2p += kstep) {
      const cpx<T> k1 = ldg_cpx(k1p);
      const cpx<T> k2 = a.single ? mk<T>(0, 0) : ldg_cpx(k2p);
      cpx<T> num = cmulc(k1, r1[idx]);
      T den = abs2(k1) + eps;
      if (!a.single) {
        num = num + cmulc(k2, r2[idx]);
        den += abs2(k2);
      }
      r1[idx] = (den != (T)0 ? recip(den) : (T)0) * num;
    }
  }
  __syncthreads();
  cpx<T>* res = fft_il<T, true, CW>(r1, a.single ? free1 : free2, a.pl, tw);
  if (vl < nv) {
    cpx<T>* dst = (cpx<T>*)a.ihat + (int64_t)fc * a.H * a.Pw2p + v0 +
                  (int64_t)(threadIdx.x / CW) * a.Pw2p + vl;
    const int64_t dstep = (int64_t)kRowStep * a.Pw2p;
    for (int idx = threadIdx.x; idx < CW * a.H; idx += kColThreads, dst += dstep) *dst = res[idx];
  }
}

struct IRowArgs {
  const cf* tw2;     // in-register inverse: w_N^(n1 k2) at [n1][k2]
  const void* ihat;  // cpx<T> [n][C][H][Pw2]
  void* latent;      // TO [n][C][H][W]
  const uint64_t* lat_tab;  // optional per-pair latent addresses ([C][H][W] each)
  int out_f64;
  int* err;          // set when a copy does not complete in time
  int n, H, W, Pw, Pw2, Pw2p, half, nbr;
  double scale;      // 1 / (Ph * Pw)
  FftPlan pl;
};

// Shared-memory layout of the inverse row pass: stage twiddles, the FFT
// buffer, two staging buffers of nbr spectrum rows (pitch Pw2p, 16-byte
// aligned); the FFT's second buffer is the consumed staging rows when a row
// fits in them (N <= Pw2p, the half-length transform), else its own.
struct IRowSmem {
  size_t tw, b0, b1, raw0, raw1, mbar, total;
  bool b1_alias;
};
__host__ __device__ inline IRowSmem irow_layout(int N, int ntw, int Pw2p, int nbr, size_t ce) {
  IRowSmem L;
  L.b1_alias = N <= Pw2p;
  size_t o = 0;
  L.tw = o;
  o += rp_align((size_t)((ntw + 1) & ~1) * ce);
  L.b0 = o;
  o += rp_align((size_t)nbr * N * ce);
  L.b1 = o;
  if (!L.b1_alias) o += rp_align((size_t)nbr * N * ce);
  L.raw0 = o;
  o += rp_align((size_t)nbr * Pw2p * ce);
  L.raw1 = o;
  o += rp_align((size_t)nbr * Pw2p * ce);
  L.mbar = o;
  o += rp_align(2 * sizeof(uint64_t));
  L.total = o;
  return L;
}

// Bulk (TMA) copies of nr spectrum rows (whole rows of pitch Pw2p, 16-byte
// aligned) into dst rows of the same pitch, completing on `bar` (thread 0).
template <typename T, class RowPtr>
__device__ __forceinline__ void stage_spec_rows_bulk(cpx<T>* dst, const RowPtr& rowp, int nr,
                                                     int Pw2p, uint64_t* bar) {
  if (threadIdx.x == 0) {
    const uint32_t bytes = (uint32_t)(Pw2p * sizeof(cpx<T>));
    mbar_expect_tx(bar, bytes * (uint32_t)nr);
    for (int i = 0; i < nr; ++i) bulk_g2s(dst + i * Pw2p, rowp(i), bytes, bar);
  }
}

// First inverse Stockham stage (Ns = 1), reading the staged spectrum rows
// directly: element m of the half-length transform is E + i O, E and O the
// even and odd parts of X[m] and conj(X[N - m]) (O with the twiddle
// exp(+2 pi i m / Pw)); for odd Pw, element m is the Hermitian extension of X.
template <typename T, int R, int NC = 0>
__device__ __forceinline__ void stage_first_spec(const cpx<T>* raw, int Pw2p, const cpx<T>* tw_w,
                                                 bool half, int Pw2, cpx<T>* out,
                                                 const FftStage& st, int N_, int nb) {
  const int Nr = NC ? NC / R : st.Nr, N = NC ? NC : N_;
  for (int idx = threadIdx.x; idx < nb * Nr; idx += blockDim.x) {
    const int b = NC ? idx / (NC / R) : st.mNr ? (int)__umulhi((unsigned)idx, st.mNr) : idx;
    const int j = idx - b * Nr;
    const cpx<T>* Xr = raw + b * Pw2p;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int m = j + r * Nr;
      if (half) {
        const cpx<T> xk = Xr[m], xc = conj(Xr[N - m]);
        const cpx<T> e = (T)0.5 * (xk + xc), d = (T)0.5 * (xk - xc);
        const cpx<T> o = conj(ldg_cpx(tw_w + m)) * d;   // exp(+2 pi i m / Pw) d
        v[r] = mk<T>(e.re - o.im, e.im + o.re);          // E + i O
      } else {
        v[r] = m < Pw2 ? Xr[m] : conj(Xr[N - m]);
      }
    }
    small_dft<T, true, R>(v);
    cpx<T>* dst = out + b * N + j * R;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r] = v[r];
  }
}

template <typename T>
__device__ __forceinline__ void first_stage_spec(const cpx<T>* raw, int Pw2p, const cpx<T>* tw_w,
                                                 bool half, int Pw2, cpx<T>* out, const FftPlan& pl,
                                                 int nb) {
  const FftStage& st = pl.st[0];
  switch (st.R) {
    case 2: stage_first_spec<T, 2>(raw, Pw2p, tw_w, half, Pw2, out, st, pl.n, nb); break;
    case 3: stage_first_spec<T, 3>(raw, Pw2p, tw_w, half, Pw2, out, st, pl.n, nb); break;
    case 4: stage_first_spec<T, 4>(raw, Pw2p, tw_w, half, Pw2, out, st, pl.n, nb); break;
    case 5: stage_first_spec<T, 5>(raw, Pw2p, tw_w, half, Pw2, out, st, pl.n, nb); break;
    case 7: stage_first_spec<T, 7>(raw, Pw2p, tw_w, half, Pw2, out, st, pl.n, nb); break;
    case 8: stage_first_spec<T, 8>(raw, Pw2p, tw_w, half, Pw2, out, st, pl.n, nb); break;
    default: stage_first_spec<T, 9>(raw, Pw2p, tw_w, half, Pw2, out, st, pl.n, nb); break;
  }
}

// Inverse complex-to-real FFT of every row, crop and scale.  A block owns the
// rows x, x + X, ... (x = blockIdx.x, X = gridDim.x) of one frame channel, nbr
// at a time, the next group's spectrum rows in flight (bulk copies on an
// mbarrier per staging buffer) while the current group is transformed.
template <typename T>
__global__ void __launch_bounds__(kRowPassThreads)
k_row_ifft(IRowArgs a, const cpx<T>* tw_w, const cpx<T>* stw) {
  extern __shared__ __align__(16) char smem[];
  const int N = a.pl.n, NB = a.nbr;
  const IRowSmem L = irow_layout(N, a.pl.ntw, a.Pw2p, NB, sizeof(cpx<T>));
  cpx<T>* tw = (cpx<T>*)(smem + L.tw);
  cpx<T>* b0 = (cpx<T>*)(smem + L.b0);
  cpx<T>* const raw0 = (cpx<T>*)(smem + L.raw0);
  cpx<T>* const raw1 = (cpx<T>*)(smem + L.raw1);
  uint64_t* bars = (uint64_t*)(smem + L.mbar);
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t par = 0u;   // bit b: phase parity of buffer b's next completion
  load_twiddles(tw, stw, a.pl.ntw);
  const int fc = blockIdx.y;
  const int x0 = blockIdx.x, X = gridDim.x;
  const int nrows = x0 < a.H ? (a.H - x0 + X - 1) / X : 0;
  const int ngroups = (nrows + NB - 1) / NB;
  auto row_of = [&](int g, int i) { return x0 + (g * NB + i) * X; };
  const cpx<T>* src = (const cpx<T>*)a.ihat + (int64_t)fc * a.H * a.Pw2p;
  void* outp = a.latent;
  int64_t obase = (int64_t)fc * a.H * a.W;
  if (a.lat_tab) {
    const int C = gridDim.y / a.n;
    outp = (void*)a.lat_tab[fc / C];
    obase = (int64_t)(fc % C) * a.H * a.W;
  }
  if (ngroups > 0)
    stage_spec_rows_bulk<T>(raw0, [&](int i) { return src + (int64_t)row_of(0, i) * a.Pw2p; },
                            min(NB, nrows), a.Pw2p, &bars[0]);
  const T sc = (T)a.scale;
  for (int g = 0; g < ngroups; ++g) {
    const int nr = min(NB, nrows - g * NB);
    if (g + 1 < ngroups) {
      const int g1 = g + 1;
      stage_spec_rows_bulk<T>((g1 & 1) ? raw1 : raw0,
                              [&](int i) { return src + (int64_t)row_of(g1, i) * a.Pw2p; },
                              min(NB, nrows - g1 * NB), a.Pw2p, &bars[g1 & 1]);
    }
    const bool arrived = mbar_wait(&bars[g & 1], (par >> (g & 1)) & 1u, kWaitLimit);
    par ^= 1u << (g & 1);
    if (__syncthreads_or(!arrived)) {
      // a copy did not complete in time: report it, wait (bounded) for the
      // other buffer's copies still in flight, and leave
      if (threadIdx.x == 0) atomicOr(a.err, 1);
      if (g + 1 < ngroups) mbar_wait(&bars[(g + 1) & 1], (par >> ((g + 1) & 1)) & 1u, kWaitLimit);
      return;
    }
    cpx<T>* const rw0 = (g & 1) ? raw1 : raw0;
    // first inverse stage straight from the staged spectrum rows into b0
    if (plan_is<CBP_ROW_PLAN>(a.pl))
      stage_first_spec<T, 9, 972>(rw0, a.Pw2p, tw_w, a.half, a.Pw2, b0, a.pl.st[0], 972, nr);
    else
      first_stage_spec<T>(rw0, a.Pw2p, tw_w, a.half, a.Pw2, b0, a.pl, nr);
    __syncthreads();
    cpx<T>* b1 = L.b1_alias ? rw0 : (cpx<T>*)(smem + L.b1);
    cpx<T>* Z = plan_is<CBP_ROW_PLAN>(a.pl) ? fft_rest_fixed<T, true, CBP_ROW_PLAN>(b0, b1, nr, tw)
                                            : fft_block<T, true>(b0, b1, a.pl, nr, tw, 1);
    for (int i = 0; i < nr; ++i) {
      const cpx<T>* z = Z + i * N;
      const int64_t ob = obase + (int64_t)row_of(g, i) * a.W;
      if (a.half && !a.out_f64 && (((ob * 4 + (uintptr_t)outp) & 7) == 0)) {
        float2* o2 = (float2*)((float*)outp + ob);
        for (int m = threadIdx.x; m < (a.W >> 1); m += blockDim.x)
          o2[m] = make_float2((float)((T)2 * sc * z[m].re), (float)((T)2 * sc * z[m].im));
        if ((a.W & 1) && threadIdx.x == 0)
          ((float*)outp)[ob + a.W - 1] = (float)((T)2 * sc * z[a.W >> 1].re);
      } else {
        for (int c = threadIdx.x; c < a.W; c += blockDim.x) {
          T v;
          if (a.half) v = (c & 1) ? (T)2 * z[c >> 1].im : (T)2 * z[c >> 1].re;
          else v = z[c].re;
          v *= sc;
          if (a.out_f64) ((double*)outp)[ob + c] = (double)v;
          else ((float*)outp)[ob + c] = (float)v;
        }
      }
    }
    // the staging rows of this group (also the FFT's scratch) are rewritten
    // by a later bulk copy: order their generic-proxy accesses before it
    fence_proxy_async();
    __syncthreads();
  }
}


// ---------------- inverse row pass with in-register transforms (float)
//
// The inverse of k_row_pass_ir for float output rows starting on 8-byte
// boundaries: per spectrum row, the half-length sequence
//   Z[k] = E + i O,  E = (X[k] + conj X[N-k]) / 2,  O = w_Pw^-k (X[k] - conj X[N-k]) / 2,
// its inverse N-point DFT z by the two-factor split (step A: per (row, k2)
// an N1-point inverse DFT over k1, twiddled by w_N^-(n1 k2); step B: per
// (row, n1) an N2-point inverse DFT over k2), then x[2m] = Re z[m],
// x[2m+1] = Im z[m], scaled by 2 / (Ph Pw) and cropped to W.  The staged
// spectrum rows are overwritten in place; two buffers of kIrRows rows, the
// next group's copy in flight while one is transformed.
struct IRowIrSmem {
  size_t raw0, raw1, mbar, total;
};
__host__ __device__ inline IRowIrSmem irow_ir_layout(int Pw2p) {
  IRowIrSmem L;
  size_t o = 0;
  L.raw0 = o;
  o += rp_align((size_t)kIrRows * Pw2p * sizeof(cf));
  L.raw1 = o;
  o += rp_align((size_t)kIrRows * Pw2p * sizeof(cf));
  L.mbar = o;
  o += rp_align(2 * sizeof(uint64_t));
  L.total = o;
  return L;
}

template <int N1, int N2>
__global__ void __launch_bounds__(kIrThreads, 2) k_row_ifft_ir(IRowArgs a, const cf* tw_w) {
  constexpr int N = N1 * N2;
  extern __shared__ __align__(16) char smem[];
  const IRowIrSmem L = irow_ir_layout(a.Pw2p);
  cf* const raw0 = (cf*)(smem + L.raw0);
  cf* const raw1 = (cf*)(smem + L.raw1);
  uint64_t* bars = (uint64_t*)(smem + L.mbar);   // one per staging buffer
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t par = 0u;   // bit b: phase parity of buffer b's next completion
  const int fc = blockIdx.y;
  const int x0 = blockIdx.x, X = gridDim.x;
  const int nrows = x0 < a.H ? (a.H - x0 + X - 1) / X : 0;
  const int ngroups = (nrows + kIrRows - 1) / kIrRows;
  auto row_of = [&](int g, int i) { return x0 + (g * kIrRows + i) * X; };
  const cf* src = (const cf*)a.ihat + (int64_t)fc * a.H * a.Pw2p;
  float* outp = (float*)a.latent + (int64_t)fc * a.H * a.W;
  const float sc2 = (float)(2.0 * a.scale);
  if (ngroups > 0)
    stage_spec_rows_bulk<float>(raw0, [&](int i) { return src + (int64_t)row_of(0, i) * a.Pw2p; },
                                min(kIrRows, nrows), a.Pw2p, &bars[0]);
  const int warp = tid >> 5, lane = tid & 31;
  for (int g = 0; g < ngroups; ++g) {
    const int nr = min(kIrRows, nrows - g * kIrRows);
    cf* const raw = (g & 1) ? raw1 : raw0;
    if (g + 1 < ngroups) {
      const int g1 = g + 1;
      stage_spec_rows_bulk<float>((g1 & 1) ? raw1 : raw0,
                                  [&](int i) { return src + (int64_t)row_of(g1, i) * a.Pw2p; },
                                  min(kIrRows, nrows - g1 * kIrRows), a.Pw2p, &bars[g1 & 1]);
    }
    const bool arrived = mbar_wait(&bars[g & 1], (par >> (g & 1)) & 1u, kWaitLimit);
    par ^= 1u << (g & 1);
    if (__syncthreads_or(!arrived)) {
      // a copy did not complete in time: report it, wait (bounded) for the
      // other buffer's copy still in flight, and leave
      if (tid == 0) atomicOr(a.err, 1);
      if (g + 1 < ngroups) mbar_wait(&bars[(g + 1) & 1], (par >> ((g + 1) & 1)) & 1u, kWaitLimit);
      return;
    }
    // ---- step A: one warp per row, lane k2
    const bool ta = warp < nr && lane < N2;
    const int k2 = lane;
    (void)CBP_CHECK(N < a.Pw2p && nr <= kIrRows && kIrRows <= kIrThreads / 32, 3);
    cf x[N1];
    if (ta) {
      const cf* X_ = raw + warp * a.Pw2p;
      const cf* tw = tw_w + k2;
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int k = k2 + N2 * k1;                 // < N
        const cf xk = X_[k], xc = conj(X_[N - k]);
        const cf e = bf_scale(0.5f, bf_add(xk, xc)), d = bf_scale(0.5f, bf_sub(xk, xc));
        const cf o = conj(ldg_cpx(tw + N2 * k1)) * d;   // w_Pw^-k d
        x[k1] = mk(e.re - o.im, e.im + o.re);       // E + i O
      }
      static_assert(N2 <= 32, "one lane per k2");
      reg_dft<true, N1>(x);
      const cf* tn = a.tw2 + k2;                    // w_N^(n1 k2) at [n1][k2]: lanes read in a row
#pragma unroll
      for (int n1 = 1; n1 < N1; ++n1) x[reg_pos<N1>(n1)] = x[reg_pos<N1>(n1)] * conj(ldg_cpx(tn + N2 * n1));
    }
    __syncthreads();
    if (ta) {
      cf* z = raw + warp * a.Pw2p + N1 * k2;
      const int sw = (k2 >> 2) & 3;
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) z[n1 ^ sw] = x[reg_pos<N1>(n1)];
    }
    __syncthreads();
    // ---- step B: per (row, n1), the N2-point inverse DFT over k2, rows out
    if (tid < nr * N1) {
      const int i = tid / N1, n1 = tid - i * N1;
      const cf* z = raw + i * a.Pw2p;
      const cf* q[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) q[c] = z + (n1 ^ c);
      cf y[N2];
#pragma unroll
      for (int kk = 0; kk < N2; ++kk) y[kk] = q[(kk >> 2) & 3][N1 * kk];
      reg_dft<true, N2>(y);
      float* o = outp + (int64_t)row_of(g, i) * a.W;
      (void)CBP_CHECK(row_of(g, i) < a.H, 4);
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        const int c = 2 * (n1 + N1 * n2);
        const cf v = y[reg_pos<N2>(n2)];
        if (c + 1 < a.W) *(float2*)(o + c) = make_float2(sc2 * v.re, sc2 * v.im);
        else if (c < a.W) o[c] = sc2 * v.re;
      }
    }
    // this buffer is rewritten by the copy issued two groups on: order its
    // generic-proxy accesses first
    fence_proxy_async();
    __syncthreads();
  }
}

template <typename T>
void run_kernel_spectra(const Plan& p, char* ws, cudaStream_t st) {
  const cpx<T>* tw_h = (const cpx<T>*)(ws + p.off_tw_h);
  const cpx<T>* tw_w = (const cpx<T>*)(ws + p.off_tw_w);
  dim3 g((p.Pw2 + kSpecCols - 1) / kSpecCols, 2, p.n);
  const size_t sm = sizeof(cpx<T>) * ((size_t)kMaxN * kSpecCols + p.Ph);
  cudaFuncSetAttribute(k_kernel_spectra<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_kernel_spectra<T><<<g, kFftThreads, sm, st>>>((const double*)(ws + p.off_kd), p.t1, p.t2, p.Ph,
                                                  p.Pw, p.Pw2, p.Pw2p, tw_h, tw_w,
                                                  (cpx<T>*)(ws + p.off_khat));
}

// Shared-memory target of the row pass: two resident blocks per SM.
constexpr size_t kRowPassSmemTarget = 112 * 1024;

template <typename T, typename In, bool FOLD, bool FFT>
void run_row_pass_t(const Plan& p, const RowPassArgs& a, int gx, int gz, char* ws,
                    cudaStream_t st) {
  const RowPassSmem L = row_pass_layout(a.pl.n, a.pl.ntw, a.wl, a.nbr, a.rw, sizeof(cpx<T>),
                                        sizeof(In), FOLD, FFT);
  cudaFuncSetAttribute(k_row_pass<T, In, FOLD, FFT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)L.total);
  k_row_pass<T, In, FOLD, FFT><<<dim3(gx, p.n * p.C, gz), kRowPassThreads, L.total, st>>>(
      a, (const cpx<T>*)(ws + p.off_tw_w), (const cpx<T>*)(ws + p.off_stw_r));
}

// The in-register row pass applies: float rows starting on 8-byte boundaries
// (strided batches; tables of per-pair addresses take the general kernel) and
// a half-length transform of 972 = 36 x 27 points.
static bool row_pass_ir_ok(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, bool fft) {
  if (!fft || p.fft_f64 || b1.f64 || !p.pw_half || p.fp_w2.n != 972 || p.M > 32 || !p.off_tw2r)
    return false;
  for (const FrameDesc* b : {&b1, &b2}) {
    if (b->tab || ((uintptr_t)b->data & 7) || (b->rs & 1) || (b->cs & 1) || (b->fs & 1)) return false;
  }
  return true;
}

template <typename T, typename In>
void run_row_pass(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                  cudaStream_t st, bool fold, bool fft) {
  RowPassArgs a;
  a.tw2 = p.off_tw2r ? (const cf*)(ws + p.off_tw2r) : nullptr;
  a.fr[0] = b1;
  a.fr[1] = b2;
  a.spec[0] = ws + p.off_spec[0];
  a.spec[1] = ws + p.off_spec[1];
  for (int k = 0; k < 2; ++k) {
    a.bins_r[k] = ws + p.off_fbr[k];
    a.bins_c[k] = ws + p.off_fbc[k];
  }
  a.bad = (int*)(ws + p.off_bad);
  a.err = (int*)(ws + p.off_err);
  a.M = p.M;
  a.fft_frames = p.single_kernel ? 1 : 2;
  a.Pw = p.Pw;
  a.Pw2 = p.Pw2;
  a.Pw2p = p.Pw2p;
  a.half = p.pw_half;
  a.pl = p.pw_half ? p.fp_w2 : p.fp_w;
  a.wl = p.W1 > p.W2 ? p.W1 : p.W2;
  constexpr int E = 16 / (int)sizeof(In);
  a.rw = ((a.wl + 2 * E + E - 1) / E) * E;
  // rows per group: the most (up to 8) that keep two blocks per SM
  a.nbr = 1;
  for (int nb = 8; nb >= 1; nb >>= 1) {
    const RowPassSmem L = row_pass_layout(a.pl.n, a.pl.ntw, a.wl, nb, a.rw, sizeof(cpx<T>),
                                          sizeof(In), fold, fft);
    if (L.total <= kRowPassSmemTarget && (!fft || (long)nb * a.pl.n <= 65535)) {
      a.nbr = nb;
      break;
    }
  }
  const int hmax = p.H1 > p.H2 ? p.H1 : p.H2;
  const int gx = fold ? p.M : (hmax + 31) / 32;
  const int gz = fold ? 2 : a.fft_frames;
  if constexpr (sizeof(T) == 4 && sizeof(In) == 4) {
    if (row_pass_ir_ok(p, b1, b2, fft)) {
      a.rw = ((2 * a.pl.n + 4 + 3) / 4) * 4;       // transform length + the 16-byte phase
      const RowIrSmem L = row_ir_layout(a.rw);
      auto kern = fold ? k_row_pass_ir<36, 27, true> : k_row_pass_ir<36, 27, false>;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
      cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      kern<<<dim3(gx, p.n * p.C, gz), kIrThreads, L.total, st>>>(a, (const cf*)(ws + p.off_tw_w));
      return;
    }
  }
  if (fold && fft) run_row_pass_t<T, In, true, true>(p, a, gx, gz, ws, st);
  else if (fft) run_row_pass_t<T, In, false, true>(p, a, gx, gz, ws, st);
  else run_row_pass_t<float, In, true, false>(p, a, gx, gz, ws, st);
}

template <typename T, bool RESID>
void run_col_deconv(const Plan& p, char* ws, cudaStream_t st) {
  ColArgs a;
  a.spec[0] = ws + p.off_spec[0];
  a.spec[1] = ws + p.off_spec[1];
  a.khat = ws + p.off_khat;
  a.ihat = ws + p.off_ihat;
  a.stw = ws + p.off_stw_h;
  a.H1 = p.H1;
  a.H2 = p.H2;
  a.H = p.H;
  a.C = p.C;
  a.Ph = p.Ph;
  a.Pw = p.Pw;
  a.Pw2 = p.Pw2;
  a.Pw2p = p.Pw2p;
  a.single = RESID ? 0 : p.single_kernel;
  a.eps = p.eps;
  a.rpart = RESID ? (double*)(ws + p.off_rpart) : nullptr;
  a.pl = p.fp_h;
  constexpr int CW = sizeof(T) == 4 ? 4 : 2;
  dim3 g((p.Pw2 + CW - 1) / CW, p.n * p.C);
  const size_t sm = sizeof(cpx<T>) * 3 * (size_t)CW * p.Ph;
  cudaFuncSetAttribute(k_col_deconv<T, CW, RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
  k_col_deconv<T, CW, RESID><<<g, kColThreads, sm, st>>>(a);
}

// Learned path: rho and the accept flag of every pair from the partial sums
// (fixed summation order).
// One CTA per pair: the pair's C * strips partial sums, reduced in a fixed
// order (deterministic), then rho and the decision.
constexpr int kGateThreads = 128;
__global__ void __launch_bounds__(kGateThreads) k_gate(const double* rpart, int n, int C, int strips,
                                                      double accept_rho, int* acc, double* rho) {
  const int f = blockIdx.x;
  const int m = C * strips;
  const double* o = rpart + (int64_t)f * m * 2;
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    num += o[2 * i];
    den += o[2 * i + 1];
  }
  __shared__ double red[2][kGateThreads / 32];
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sn = 0.0, sd = 0.0;
    for (int w = 0; w < kGateThreads / 32; ++w) {
      sn += red[0][w];
      sd += red[1][w];
    }
    const double r = sd > 0.0 ? sqrt(sn / sd) : INFINITY;
    rho[f] = r;
    acc[f] = r <= accept_rho ? 1 : 0;
  }
}

template <typename T>
void run_row_ifft(const Plan& p, char* ws, void* latent, int out_f64, cudaStream_t st,
                  const uint64_t* lat_tab) {
  const FftPlan& plw = p.pw_half ? p.fp_w2 : p.fp_w;
  IRowArgs a;
  a.tw2 = p.off_tw2r ? (const cf*)(ws + p.off_tw2r) + 972 : nullptr;
  a.ihat = ws + p.off_ihat;
  a.latent = latent;
  a.lat_tab = lat_tab;
  a.out_f64 = out_f64;
  a.err = (int*)(ws + p.off_err);
  a.n = p.n;
  a.H = p.H;
  a.W = p.W;
  a.Pw = p.Pw;
  a.Pw2 = p.Pw2;
  a.Pw2p = p.Pw2p;
  a.half = p.pw_half;
  a.scale = 1.0 / ((double)p.Ph * (double)p.Pw);
  a.pl = plw;
  a.nbr = 1;
  for (int nb = 8; nb >= 1; nb >>= 1) {
    if (irow_layout(plw.n, plw.ntw, p.Pw2p, nb, sizeof(cpx<T>)).total <= kRowPassSmemTarget &&
        (long)nb * plw.n <= 65535) {
      a.nbr = nb;
      break;
    }
  }
  dim3 g((p.H + 31) / 32, p.n * p.C);
  if constexpr (sizeof(T) == 4) {
    // in-register transforms: float output rows on 8-byte boundaries, 972 = 36 x 27
    if (p.pw_half && plw.n == 972 && !out_f64 && !lat_tab && (p.W % 2) == 0 &&
        ((uintptr_t)latent & 7) == 0 && p.off_tw2r) {
      const size_t smi = irow_ir_layout(p.Pw2p).total;
      cudaFuncSetAttribute(k_row_ifft_ir<36, 27>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smi);
      cudaFuncSetAttribute(k_row_ifft_ir<36, 27>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      k_row_ifft_ir<36, 27><<<g, kIrThreads, smi, st>>>(a, (const cf*)(ws + p.off_tw_w));
      return;
    }
  }
  const size_t sm = irow_layout(plw.n, plw.ntw, p.Pw2p, a.nbr, sizeof(cpx<T>)).total;
  cudaFuncSetAttribute(k_row_ifft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_row_ifft<T><<<g, kRowPassThreads, sm, st>>>(a, (const cpx<T>*)(ws + p.off_tw_w),
                                                (const cpx<T>*)(ws + p.off_stw_r));
}

}  // namespace

// Transposed twiddle tables of a two-factor split N = A B:
// out[b A + a] = w_N^(a b) and out[A B + a B + b] = w_N^(a b), a < A, b < B.
__global__ void k_twiddles_2f(cf* out, int A, int B) {
  const int N = A * B;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const int b = e / A, a = e % A;
    double sn, cs;
    sincospi(-2.0 * (double)((a * b) % N) / (double)N, &sn, &cs);
    const cf w = mk((float)cs, (float)sn);
    out[b * A + a] = w;
    out[N + a * B + b] = w;
  }
}

template <typename T>
void run_twiddles(const Plan& p, char* ws, cudaStream_t st) {
  if (p.off_tw2r) k_twiddles_2f<<<4, 256, 0, st>>>((cf*)(ws + p.off_tw2r), 36, 27);
  if (p.off_tw2c) k_twiddles_2f<<<5, 256, 0, st>>>((cf*)(ws + p.off_tw2c), 32, 35);
  k_twiddles<T><<<(p.Ph + 255) / 256, 256, 0, st>>>((cpx<T>*)(ws + p.off_tw_h), p.Ph);
  k_twiddles<T><<<(p.Pw + 255) / 256, 256, 0, st>>>((cpx<T>*)(ws + p.off_tw_w), p.Pw);
  const FftPlan& plw = p.pw_half ? p.fp_w2 : p.fp_w;
  k_stage_twiddles<T><<<(p.Ph + 255) / 256, 256, 0, st>>>(p.fp_h, (cpx<T>*)(ws + p.off_stw_h));
  k_stage_twiddles<T><<<(plw.n + 255) / 256, 256, 0, st>>>(plw, (cpx<T>*)(ws + p.off_stw_r));
}

void init_twiddles(const Plan& p, char* ws, cudaStream_t st) {
  if (p.fft_f64) run_twiddles<double>(p, ws, st);
  else run_twiddles<float>(p, ws, st);
}

void launch_kernel_spectra(const Plan& p, char* ws, cudaStream_t st) {
  if (p.fft_f64) run_kernel_spectra<double>(p, ws, st);
  else run_kernel_spectra<float>(p, ws, st);
}

void launch_row_pass(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                     cudaStream_t st, bool fold, bool fft) {
  if (!fold && !fft) return;
  if (fft && p.fft_f64) {
    if (b1.f64) run_row_pass<double, double>(p, b1, b2, ws, st, fold, fft);
    else run_row_pass<double, float>(p, b1, b2, ws, st, fold, fft);
  } else {
    if (b1.f64) run_row_pass<float, double>(p, b1, b2, ws, st, fold, fft);
    else run_row_pass<float, float>(p, b1, b2, ws, st, fold, fft);
  }
}

size_t row_pass_min_smem(const Plan& p) {
  const FftPlan& pl = p.pw_half ? p.fp_w2 : p.fp_w;
  const int wl = p.W1 > p.W2 ? p.W1 : p.W2;
  const size_t ce = p.fft_f64 ? 16 : 8;
  const int rw = ((wl + 4 + 1) / 2) * 2;   // staging pitch for 8-byte elements (the widest)
  const size_t fwd = row_pass_layout(pl.n, pl.ntw, wl, 1, rw, ce, 8, true, true).total;
  const size_t inv = irow_layout(pl.n, pl.ntw, p.Pw2p, 1, ce).total;
  return fwd > inv ? fwd : inv;
}

void launch_col_deconv(const Plan& p, char* ws, cudaStream_t st) {
  if (p.col_fused) launch_col_deconv_fused(p, ws, st);
  else if (p.fft_f64) run_col_deconv<double, false>(p, ws, st);
  else run_col_deconv<float, false>(p, ws, st);
}

void launch_row_ifft(const Plan& p, char* ws, void* latent, int out_f64, cudaStream_t st,
                     const uint64_t* lat_tab) {
  if (p.fft_f64) run_row_ifft<double>(p, ws, latent, out_f64, st, lat_tab);
  else run_row_ifft<float>(p, ws, latent, out_f64, st, lat_tab);
}

void launch_gate(const Plan& p, char* ws, cudaStream_t st, int strips) {
  k_gate<<<p.n, kGateThreads, 0, st>>>((const double*)(ws + p.off_rpart), p.n, p.C, strips,
                                            p.accept_rho, (int*)(ws + p.off_acc),
                                            (double*)(ws + p.off_rho));
}

void launch_residual_gate(const Plan& p, char* ws, cudaStream_t st) {
  if (p.fft_f64) run_col_deconv<double, true>(p, ws, st);
  else run_col_deconv<float, true>(p, ws, st);
  launch_gate(p, ws, st, p.col_strips);
}

bool set_tx_extra(uint32_t bytes) {
#ifdef CBP_CHECKS
  return cudaMemcpyToSymbol(cbp_tx_extra, &bytes, sizeof bytes) == cudaSuccess;
#else
  (void)bytes;
  return false;
#endif
}

}  // namespace cbp
