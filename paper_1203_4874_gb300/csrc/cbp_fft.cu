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
#include "cbp_internal.h"

namespace cbp {
namespace {

constexpr int kFftThreads = 256;

// cos / sin (2 pi j / R) for the odd radices
__constant__ double kC3[3] = {1.0, -0.5, -0.5};
__constant__ double kS3[3] = {0.0, 0.86602540378443864676, -0.86602540378443864676};
__constant__ double kC5[5] = {1.0, 0.30901699437494742410, -0.80901699437494742410,
                              -0.80901699437494742410, 0.30901699437494742410};
__constant__ double kS5[5] = {0.0, 0.95105651629515357212, 0.58778525229247312917,
                              -0.58778525229247312917, -0.95105651629515357212};
__constant__ double kC7[7] = {1.0, 0.62348980185873353053, -0.22252093395631440429,
                              -0.90096886790241912624, -0.90096886790241912624,
                              -0.22252093395631440429, 0.62348980185873353053};
__constant__ double kS7[7] = {0.0, 0.78183148246802980871, 0.97492791218182360702,
                              0.43388373911755812048, -0.43388373911755812048,
                              -0.97492791218182360702, -0.78183148246802980871};

// In-register DFT of size R; sgn = -1 forward, +1 inverse (unnormalised).
template <typename T, int R>
__device__ __forceinline__ void small_dft(cpx<T>* v, T sgn) {
  if constexpr (R == 2) {
    cpx<T> a = v[0] + v[1], b = v[0] - v[1];
    v[0] = a;
    v[1] = b;
  } else if constexpr (R == 4) {
    cpx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], d = v[1] - v[3];
    cpx<T> t3 = mk<T>(-sgn * d.im, sgn * d.re);  // sgn * i * d
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  } else {
    const double* C = R == 3 ? kC3 : (R == 5 ? kC5 : kC7);
    const double* S = R == 3 ? kS3 : (R == 5 ? kS5 : kS7);
    constexpr int H = (R - 1) / 2;
    cpx<T> a[H], b[H];
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      a[m - 1] = v[m] + v[R - m];
      b[m - 1] = v[m] - v[R - m];
    }
    cpx<T> x0 = v[0];
    cpx<T> s0 = x0;
#pragma unroll
    for (int m = 0; m < H; ++m) s0 = s0 + a[m];
    v[0] = s0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      cpx<T> re = x0, im = mk<T>(0, 0);
#pragma unroll
      for (int m = 1; m <= H; ++m) {
        const int j = (k * m) % R;
        const T c = (T)C[j], s = (T)S[j];
        re = re + c * a[m - 1];
        im = im + s * b[m - 1];
      }
      // X[k] = re + sgn*i*im ; X[R-k] = re - sgn*i*im
      cpx<T> si = mk<T>(-sgn * im.im, sgn * im.re);
      v[k] = re + si;
      v[R - k] = re - si;
    }
  }
}

// One Stockham stage of radix R over `nb` transforms of length N stored with
// stride N (in -> out).  Twiddles w_N^e = tw[e * tstride] (tw of length N * tstride).
template <typename T, int R>
__device__ void stockham_stage(const cpx<T>* in, cpx<T>* out, int N, int Ns, int nb,
                               const cpx<T>* tw, int tstride, T sgn) {
  const int Nr = N / R;
  const int estep = N / (Ns * R);
  for (int idx = threadIdx.x; idx < nb * Nr; idx += blockDim.x) {
    const int b = idx / Nr, j = idx - b * Nr;
    const cpx<T>* src = in + (int64_t)b * N;
    cpx<T>* dst = out + (int64_t)b * N;
    const int k = j % Ns;
    cpx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * Nr];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cpx<T> w = tw[(int64_t)k * r * estep * tstride];
      if (sgn > 0) w.im = -w.im;
      v[r] = v[r] * w;
    }
    small_dft<T, R>(v, sgn);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
  }
}

// Full batched FFT in shared memory; returns the buffer holding the result
// (a or b).  All threads of the block must call it.
template <typename T>
__device__ cpx<T>* fft_block(cpx<T>* a, cpx<T>* b, const FftPlan& pl, int nb,
                             const cpx<T>* tw, int tstride, T sgn) {
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 2: stockham_stage<T, 2>(a, b, pl.n, Ns, nb, tw, tstride, sgn); break;
      case 3: stockham_stage<T, 3>(a, b, pl.n, Ns, nb, tw, tstride, sgn); break;
      case 4: stockham_stage<T, 4>(a, b, pl.n, Ns, nb, tw, tstride, sgn); break;
      case 5: stockham_stage<T, 5>(a, b, pl.n, Ns, nb, tw, tstride, sgn); break;
      default: stockham_stage<T, 7>(a, b, pl.n, Ns, nb, tw, tstride, sgn); break;
    }
    __syncthreads();
    cpx<T>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
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
// kv[p][v] = sum_q K[p][q] w_Pw^{vq} (double), then K^[u][v] = sum_p kv[p][v] w_Ph^{up}.
template <typename T>
__global__ void __launch_bounds__(kFftThreads)
k_kernel_spectra(const double* kd, int t1, int t2, int Ph, int Pw, int Pw2, const cpx<T>* tw_h,
                 const cpx<T>* tw_w, cpx<T>* khat) {
  constexpr int CW = 16;
  __shared__ cpx<T> kv[kMaxN * CW];
  const int k = blockIdx.y, f = blockIdx.z;
  const int t = k ? t2 : t1;
  const double* K = kd + (int64_t)f * (t1 * t1 + t2 * t2) + (k ? t1 * t1 : 0);
  const int v0 = blockIdx.x * CW;
  for (int idx = threadIdx.x; idx < t * CW; idx += blockDim.x) {
    const int p = idx / CW, vl = idx % CW, v = v0 + vl;
    cd acc = mk(0.0, 0.0);
    if (v < Pw2) {
      int e = 0;                              // (v q) mod Pw, incrementally
      for (int q = 0; q < t; ++q) {
        acc = acc + K[p * t + q] * cvt<double>(tw_w[e]);
        e += v;
        if (e >= Pw) e -= Pw;
      }
    }
    kv[idx] = cvt<T>(acc);
  }
  __syncthreads();
  cpx<T>* out = khat + ((int64_t)f * 2 + k) * Ph * Pw2;
  for (int idx = threadIdx.x; idx < Ph * CW; idx += blockDim.x) {
    const int u = idx / CW, vl = idx % CW, v = v0 + vl;
    if (v >= Pw2) continue;
    cpx<T> acc = mk<T>(0, 0);
    int e = 0;                                // (u p) mod Ph, incrementally
    for (int p = 0; p < t; ++p) {
      cfma(acc, kv[p * CW + vl], tw_h[e]);
      e += u;
      if (e >= Ph) e -= Ph;
    }
    out[(int64_t)u * Pw2 + v] = acc;
  }
}

struct RowArgs {
  FrameDesc fr[2];
  void* spec[2];     // cpx<T> [n][C][H_Bk][Pw2]
  int Pw, Pw2, half;
  FftPlan pl;        // plan of Pw/2 (half) or Pw
};

// Forward real-to-complex FFT of every row of B1 and B2.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_row_fft(RowArgs a, const cpx<T>* tw_w) {
  extern __shared__ __align__(16) char smem[];
  const int N = a.pl.n;
  cpx<T>* b0 = (cpx<T>*)smem;
  cpx<T>* b1 = b0 + N;
  const FrameDesc& fr = a.fr[blockIdx.z];
  const int fc = blockIdx.y, f = fc / fr.c, ch = fc % fr.c;
  const int rows_per = (fr.h + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows_per, r1 = min(fr.h, r0 + rows_per);
  cpx<T>* spec = (cpx<T>*)a.spec[blockIdx.z] + (int64_t)fc * fr.h * a.Pw2;
  for (int r = r0; r < r1; ++r) {
    const void* fb = frame_base(fr, f);
    const int64_t base = (int64_t)ch * fr.cs + (int64_t)r * fr.rs;
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
      if (a.half) {
        const int c0 = 2 * m, c1 = 2 * m + 1;
        T x0 = c0 < fr.w ? ld_frame<T>(fb, base + c0, fr.f64) : (T)0;
        T x1 = c1 < fr.w ? ld_frame<T>(fb, base + c1, fr.f64) : (T)0;
        b0[m] = mk<T>(x0, x1);
      } else {
        b0[m] = mk<T>(m < fr.w ? ld_frame<T>(fb, base + m, fr.f64) : (T)0, (T)0);
      }
    }
    __syncthreads();
    cpx<T>* Z = fft_block<T>(b0, b1, a.pl, 1, tw_w, a.half ? 2 : 1, (T)-1);
    cpx<T>* dst = spec + (int64_t)r * a.Pw2;
    for (int k = threadIdx.x; k < a.Pw2; k += blockDim.x) {
      if (a.half) {
        const cpx<T> zk = Z[k % N], zc = conj(Z[(N - k) % N]);
        const cpx<T> e = (T)0.5 * (zk + zc), d = (T)0.5 * (zk - zc);
        const cpx<T> w = tw_w[k];                 // exp(-2 pi i k / Pw)
        const cpx<T> wd = w * d;                  // X = e - i * w * d
        dst[k] = mk<T>(e.re + wd.im, e.im - wd.re);
      } else {
        dst[k] = Z[k];
      }
    }
    __syncthreads();
  }
}

struct ColArgs {
  void* spec[2];      // cpx<T> [n][C][H_Bk][Pw2]
  const void* khat;   // cpx<T> [n][2][Ph][Pw2]
  void* ihat;         // cpx<T> [n][C][H][Pw2]
  int H1, H2, H, C, Ph, Pw2, single;
  double eps;
  FftPlan pl;         // plan of Ph
};

// Column FFTs of both spectra, dual-kernel formula, inverse column FFT.
template <typename T, int CW>
__global__ void __launch_bounds__(kFftThreads) k_col_deconv(ColArgs a, const cpx<T>* tw_h) {
  extern __shared__ __align__(16) char smem[];
  const int Ph = a.Ph;
  cpx<T>* buf[3];
  for (int i = 0; i < 3; ++i) buf[i] = (cpx<T>*)smem + (int64_t)i * CW * Ph;
  const int fc = blockIdx.y, f = fc / a.C;
  const int v0 = blockIdx.x * CW;
  const int nv = min(CW, a.Pw2 - v0);
  auto load = [&](cpx<T>* dst, int k) {
    const int Hk = k ? a.H2 : a.H1;
    const cpx<T>* src = (const cpx<T>*)a.spec[k] + (int64_t)fc * Hk * a.Pw2 + v0;
    for (int idx = threadIdx.x; idx < CW * Ph; idx += blockDim.x) {
      const int u = idx / CW, vl = idx % CW;
      dst[vl * Ph + u] = (u < Hk && vl < nv) ? src[(int64_t)u * a.Pw2 + vl] : mk<T>(0, 0);
    }
    __syncthreads();
  };
  const cpx<T>* K1 = (const cpx<T>*)a.khat + ((int64_t)f * 2 + 0) * Ph * a.Pw2 + v0;
  const cpx<T>* K2 = (const cpx<T>*)a.khat + ((int64_t)f * 2 + 1) * Ph * a.Pw2 + v0;
  load(buf[0], 0);
  cpx<T>* r1 = fft_block<T>(buf[0], buf[1], a.pl, CW, tw_h, 1, (T)-1);
  cpx<T>* free1 = r1 == buf[0] ? buf[1] : buf[0];
  cpx<T>* r2 = nullptr;
  cpx<T>* free2 = nullptr;
  if (!a.single) {
    load(buf[2], 1);
    r2 = fft_block<T>(buf[2], free1, a.pl, CW, tw_h, 1, (T)-1);
    free2 = r2 == buf[2] ? free1 : buf[2];
  }
  const T eps = (T)a.eps;
  for (int idx = threadIdx.x; idx < CW * Ph; idx += blockDim.x) {
    const int u = idx / CW, vl = idx % CW;
    if (vl >= nv) continue;
    const cpx<T> k1 = K1[(int64_t)u * a.Pw2 + vl];
    cpx<T> num = cmulc(k1, r1[vl * Ph + u]);
    T den = abs2(k1) + eps;
    if (!a.single) {
      const cpx<T> k2 = K2[(int64_t)u * a.Pw2 + vl];
      num = num + cmulc(k2, r2[vl * Ph + u]);
      den += abs2(k2);
    }
    const T inv = den != (T)0 ? (T)1 / den : (T)0;
    r1[vl * Ph + u] = inv * num;
  }
  __syncthreads();
  cpx<T>* res = fft_block<T>(r1, a.single ? free1 : free2, a.pl, CW, tw_h, 1, (T)1);
  cpx<T>* dst = (cpx<T>*)a.ihat + (int64_t)fc * a.H * a.Pw2 + v0;
  for (int idx = threadIdx.x; idx < CW * a.H; idx += blockDim.x) {
    const int u = idx / CW, vl = idx % CW;
    if (vl < nv) dst[(int64_t)u * a.Pw2 + vl] = res[vl * Ph + u];
  }
}

struct IRowArgs {
  const void* ihat;  // cpx<T> [n][C][H][Pw2]
  void* latent;      // TO [n][C][H][W]
  const uint64_t* lat_tab;  // optional per-pair latent addresses ([C][H][W] each)
  int out_f64;
  int n, H, W, Pw, Pw2, half;
  double scale;      // 1 / (Ph * Pw)
  FftPlan pl;
};

// Inverse complex-to-real FFT of every row, crop and scale.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_row_ifft(IRowArgs a, const cpx<T>* tw_w) {
  extern __shared__ __align__(16) char smem[];
  const int N = a.pl.n;
  cpx<T>* b0 = (cpx<T>*)smem;
  cpx<T>* b1 = b0 + N;
  const int fc = blockIdx.y;
  const int rows_per = (a.H + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * rows_per, r1 = min(a.H, r0 + rows_per);
  const cpx<T>* src = (const cpx<T>*)a.ihat + (int64_t)fc * a.H * a.Pw2;
  for (int r = r0; r < r1; ++r) {
    const cpx<T>* X = src + (int64_t)r * a.Pw2;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      if (a.half) {
        const cpx<T> xk = X[k], xc = conj(X[N - k]);
        const cpx<T> e = (T)0.5 * (xk + xc), d = (T)0.5 * (xk - xc);
        const cpx<T> w = conj(tw_w[k]);        // exp(+2 pi i k / Pw)
        const cpx<T> o = w * d;
        b0[k] = mk<T>(e.re - o.im, e.im + o.re);   // E + i O
      } else {
        b0[k] = k < a.Pw2 ? X[k] : conj(X[N - k]);
      }
    }
    __syncthreads();
    cpx<T>* z = fft_block<T>(b0, b1, a.pl, 1, tw_w, a.half ? 2 : 1, (T)1);
    int64_t ob = ((int64_t)fc * a.H + r) * a.W;
    void* outp = a.latent;
    if (a.lat_tab) {
      const int C = gridDim.y / a.n;
      outp = (void*)a.lat_tab[fc / C];
      ob = ((int64_t)(fc % C) * a.H + r) * a.W;
    }
    const T sc = (T)a.scale;
    for (int c = threadIdx.x; c < a.W; c += blockDim.x) {
      T v;
      if (a.half) v = (c & 1) ? (T)2 * z[c >> 1].im : (T)2 * z[c >> 1].re;
      else v = z[c].re;
      v *= sc;
      if (a.out_f64) ((double*)outp)[ob + c] = (double)v;
      else ((float*)outp)[ob + c] = (float)v;
    }
    __syncthreads();
  }
}

template <typename T>
void run_kernel_spectra(const Plan& p, char* ws, cudaStream_t st) {
  const cpx<T>* tw_h = (const cpx<T>*)(ws + p.off_tw_h);
  const cpx<T>* tw_w = (const cpx<T>*)(ws + p.off_tw_w);
  dim3 g((p.Pw2 + 15) / 16, 2, p.n);
  k_kernel_spectra<T><<<g, kFftThreads, 0, st>>>((const double*)(ws + p.off_kd), p.t1, p.t2, p.Ph,
                                                 p.Pw, p.Pw2, tw_h, tw_w,
                                                 (cpx<T>*)(ws + p.off_khat));
}

template <typename T>
void run_row_fft(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                 cudaStream_t st) {
  const FftPlan& plw = p.pw_half ? p.fp_w2 : p.fp_w;
  RowArgs a;
  a.fr[0] = b1;
  a.fr[1] = b2;
  a.spec[0] = ws + p.off_spec[0];
  a.spec[1] = ws + p.off_spec[1];
  a.Pw = p.Pw;
  a.Pw2 = p.Pw2;
  a.half = p.pw_half;
  a.pl = plw;
  const int hmax = p.H1 > p.H2 ? p.H1 : p.H2;
  const int chunks = (hmax + 7) / 8;
  dim3 g(chunks, p.n * p.C, p.single_kernel ? 1 : 2);
  const size_t sm = 2 * sizeof(cpx<T>) * plw.n;
  cudaFuncSetAttribute(k_row_fft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_row_fft<T><<<g, kFftThreads, sm, st>>>(a, (const cpx<T>*)(ws + p.off_tw_w));
}

template <typename T>
void run_col_deconv(const Plan& p, char* ws, cudaStream_t st) {
  ColArgs a;
  a.spec[0] = ws + p.off_spec[0];
  a.spec[1] = ws + p.off_spec[1];
  a.khat = ws + p.off_khat;
  a.ihat = ws + p.off_ihat;
  a.H1 = p.H1;
  a.H2 = p.H2;
  a.H = p.H;
  a.C = p.C;
  a.Ph = p.Ph;
  a.Pw2 = p.Pw2;
  a.single = p.single_kernel;
  a.eps = p.eps;
  a.pl = p.fp_h;
  constexpr int CW = sizeof(T) == 4 ? 4 : 2;
  dim3 g((p.Pw2 + CW - 1) / CW, p.n * p.C);
  const size_t sm = 3 * sizeof(cpx<T>) * CW * p.Ph;
  cudaFuncSetAttribute(k_col_deconv<T, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_col_deconv<T, CW><<<g, kFftThreads, sm, st>>>(a, (const cpx<T>*)(ws + p.off_tw_h));
}

template <typename T>
void run_row_ifft(const Plan& p, char* ws, void* latent, int out_f64, cudaStream_t st,
                  const uint64_t* lat_tab) {
  const FftPlan& plw = p.pw_half ? p.fp_w2 : p.fp_w;
  IRowArgs a;
  a.ihat = ws + p.off_ihat;
  a.latent = latent;
  a.lat_tab = lat_tab;
  a.n = p.n;
  a.out_f64 = out_f64;
  a.H = p.H;
  a.W = p.W;
  a.Pw = p.Pw;
  a.Pw2 = p.Pw2;
  a.half = p.pw_half;
  a.scale = 1.0 / ((double)p.Ph * (double)p.Pw);
  a.pl = plw;
  dim3 g((p.H + 7) / 8, p.n * p.C);
  const size_t sm = 2 * sizeof(cpx<T>) * plw.n;
  cudaFuncSetAttribute(k_row_ifft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_row_ifft<T><<<g, kFftThreads, sm, st>>>(a, (const cpx<T>*)(ws + p.off_tw_w));
}

}  // namespace

void init_twiddles(const Plan& p, char* ws, cudaStream_t st) {
  if (p.fft_f64) {
    k_twiddles<double><<<(p.Ph + 255) / 256, 256, 0, st>>>((cd*)(ws + p.off_tw_h), p.Ph);
    k_twiddles<double><<<(p.Pw + 255) / 256, 256, 0, st>>>((cd*)(ws + p.off_tw_w), p.Pw);
  } else {
    k_twiddles<float><<<(p.Ph + 255) / 256, 256, 0, st>>>((cf*)(ws + p.off_tw_h), p.Ph);
    k_twiddles<float><<<(p.Pw + 255) / 256, 256, 0, st>>>((cf*)(ws + p.off_tw_w), p.Pw);
  }
}

void launch_kernel_spectra(const Plan& p, char* ws, cudaStream_t st) {
  if (p.fft_f64) run_kernel_spectra<double>(p, ws, st);
  else run_kernel_spectra<float>(p, ws, st);
}

void launch_row_fft(const Plan& p, const FrameDesc& b1, const FrameDesc& b2, char* ws,
                    cudaStream_t st) {
  if (p.fft_f64) run_row_fft<double>(p, b1, b2, ws, st);
  else run_row_fft<float>(p, b1, b2, ws, st);
}

void launch_col_deconv(const Plan& p, char* ws, cudaStream_t st) {
  if (p.fft_f64) run_col_deconv<double>(p, ws, st);
  else run_col_deconv<float>(p, ws, st);
}

void launch_row_ifft(const Plan& p, char* ws, void* latent, int out_f64, cudaStream_t st,
                     const uint64_t* lat_tab) {
  if (p.fft_f64) run_row_ifft<double>(p, ws, latent, out_f64, st, lat_tab);
  else run_row_ifft<float>(p, ws, latent, out_f64, st, lat_tab);
}

}  // namespace cbp
