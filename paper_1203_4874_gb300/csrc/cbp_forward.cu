// Forward model of Eq. 1 on the device (the camera side of Section 3):
// B = L (x) K + N, full 2D convolution per channel plus Gaussian noise, and a
// blob-latent synthesiser.  Random numbers come from Philox-4x32-10 (Salmon,
// Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011):
// counter = (element index lo, element index hi, stream, 0), key = seed.
#include "cbp_common.cuh"
#include "cbp_internal.h"
#include "cbp_philox.cuh"

namespace cbp {

CBP_CHECKS_TU(kChkForward)

namespace {

// Uniform in (0, 1] from 32 bits.
__device__ __forceinline__ double u01(uint32_t v) { return ((double)v + 1.0) * 2.3283064365386963e-10; }

// Standard normal number `idx` of stream `stream` (Box-Muller on one Philox block).
__device__ __forceinline__ double normal_at(uint64_t seed, uint64_t idx, uint32_t stream) {
  U4 c = {(uint32_t)idx, (uint32_t)(idx >> 32), stream, 0u};
  U4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = u01(r.x), u2 = u01(r.y);
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// The same normal number in single precision (float frames).
__device__ __forceinline__ float normal_at_f(uint64_t seed, uint64_t idx, uint32_t stream) {
  U4 c = {(uint32_t)idx, (uint32_t)(idx >> 32), stream, 0u};
  U4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u1 = ((float)(r.x >> 8) + 1.0f) * 5.9604644775390625e-8f;   // (0, 1], 24 bits
  const float u2 = ((float)(r.y >> 8) + 1.0f) * 5.9604644775390625e-8f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

template <typename T> __device__ __forceinline__ T normal_t(uint64_t seed, uint64_t idx, uint32_t stream);
template <> __device__ __forceinline__ double normal_t<double>(uint64_t s, uint64_t i, uint32_t st) {
  return normal_at(s, i, st);
}
template <> __device__ __forceinline__ float normal_t<float>(uint64_t s, uint64_t i, uint32_t st) {
  return normal_at_f(s, i, st);
}

__device__ __forceinline__ double uniform_at(uint64_t seed, uint64_t idx, uint32_t stream) {
  U4 c = {(uint32_t)idx, (uint32_t)(idx >> 32), stream, 0u};
  U4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return u01(r.x);
}

constexpr int kTile = 32;

// out[f][ch][r][c] = sum_{p,q} L[r-p][c-q] K[f][p][q] (+ noise), r < h+t-1, c < w+t-1,
// accumulated in the frame precision (double frames: double, float frames:
// float -- the data only has to be Eq. 1 to the precision it is stored in).
template <typename T>
__global__ void __launch_bounds__(kTile * 8)
k_forward_blur(const T* lat, int c, int h, int w, const double* kern, int t, double sigma,
               uint64_t seed, T* out) {
  extern __shared__ __align__(16) char smem[];
  const int hb = h + t - 1, wb = w + t - 1;
  const int fc = blockIdx.z, f = fc / c;
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  const int th = kTile + t - 1;
  T* K = (T*)smem;                           // t*t
  T* tile = (T*)(smem + ((t * t * sizeof(double) + 15) & ~size_t(15)));
  for (int i = threadIdx.x; i < t * t; i += blockDim.x) K[i] = (T)kern[(int64_t)f * t * t + i];
  const T* L = lat + (int64_t)fc * h * w;
  // tile[y][x] = L[r0 - (t-1) + y][c0 - (t-1) + x]
  for (int i = threadIdx.x; i < th * th; i += blockDim.x) {
    const int y = i / th, x = i % th;
    const int ly = r0 - (t - 1) + y, lx = c0 - (t - 1) + x;
    tile[i] = (ly >= 0 && ly < h && lx >= 0 && lx < w) ? L[(int64_t)ly * w + lx] : (T)0;
  }
  __syncthreads();
  const int tx = threadIdx.x % kTile, ty0 = threadIdx.x / kTile;
  for (int ty = ty0; ty < kTile; ty += blockDim.x / kTile) {
    const int r = r0 + ty, col = c0 + tx;
    if (r >= hb || col >= wb) continue;
    T acc = 0;
    for (int p = 0; p < t; ++p)
      for (int q = 0; q < t; ++q)
        acc = fma(K[p * t + q], tile[(ty + t - 1 - p) * th + (tx + t - 1 - q)], acc);
    const int64_t oi = ((int64_t)fc * hb + r) * wb + col;
    if (sigma > 0) acc += (T)sigma * normal_t<T>(seed, (uint64_t)oi, 1u);
    out[oi] = acc;
  }
}

// The same convolution for float frames with the kernel size fixed at compile
// time (T <= 17): a block makes 64 rows x 32 columns of output; a thread keeps
// eight consecutive output rows of one column and, for each kernel column q,
// the T + 7 input values they need in registers, so each shared-memory load
// feeds about four multiply-adds.  Sums in float, in the order p = T-1 .. 0
// for every q (as the general kernel's per-output order differs, results
// agree to float rounding, not bitwise).
constexpr int kBlurRows = 8;          // output rows per thread
constexpr int kBlurTileR = 8 * kBlurRows;
template <int T>
__global__ void __launch_bounds__(256)
k_forward_blur_rb(const float* lat, int c, int h, int w, const double* kern, double sigma,
                  uint64_t seed, float* out) {
  __shared__ float K[T * T];
  __shared__ float tile[(kBlurTileR + T - 1) * (32 + T - 1)];
  constexpr int TW = 32 + T - 1, TH = kBlurTileR + T - 1;
  const int hb = h + T - 1, wb = w + T - 1;
  const int fc = blockIdx.z, f = fc / c;
  const int r0 = blockIdx.y * kBlurTileR, c0 = blockIdx.x * 32;
  for (int i = threadIdx.x; i < T * T; i += blockDim.x) K[i] = (float)kern[(int64_t)f * T * T + i];
  const float* L = lat + (int64_t)fc * h * w;
  for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
    const int y = i / TW, x = i - y * TW;
    const int ly = r0 - (T - 1) + y, lx = c0 - (T - 1) + x;
    tile[i] = (ly >= 0 && ly < h && lx >= 0 && lx < w) ? L[(int64_t)ly * w + lx] : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[kBlurRows];
#pragma unroll
  for (int i = 0; i < kBlurRows; ++i) acc[i] = 0.f;
  // out[r][col] = sum_{p,q} K[p][q] tile[(r - r0) + T-1-p][(col - c0) + T-1-q]
  for (int q = 0; q < T; ++q) {
    float v[kBlurRows + T - 1];
    const float* col = tile + (ty * kBlurRows) * TW + tx + T - 1 - q;
    (void)CBP_CHECK((ty * kBlurRows + kBlurRows + T - 2) * TW + tx + T - 1 - q < TH * TW, 0);
#pragma unroll
    for (int j = 0; j < kBlurRows + T - 1; ++j) v[j] = col[j * TW];
#pragma unroll
    for (int p = 0; p < T; ++p) {
      const float kv = K[p * T + q];
#pragma unroll
      for (int i = 0; i < kBlurRows; ++i) acc[i] = fmaf(kv, v[i + T - 1 - p], acc[i]);
    }
  }
  const int colo = c0 + tx;
  if (colo >= wb) return;
#pragma unroll
  for (int i = 0; i < kBlurRows; ++i) {
    const int r = r0 + ty * kBlurRows + i;
    if (r >= hb) break;
    const int64_t oi = ((int64_t)fc * hb + r) * wb + colo;
    float a = acc[i];
    if (sigma > 0) a += (float)sigma * normal_at_f(seed, (uint64_t)oi, 1u);
    out[oi] = a;
  }
}

template <int T>
void launch_blur_rb(const float* lat, int n, int c, int h, int w, const double* kern, double sigma,
                    uint64_t seed, float* out, cudaStream_t st) {
  const int hb = h + T - 1, wb = w + T - 1;
  dim3 g((wb + 31) / 32, (hb + kBlurTileR - 1) / kBlurTileR, n * c);
  k_forward_blur_rb<T><<<g, 256, 0, st>>>(lat, c, h, w, kern, sigma, seed, out);
}

// Blob latent: L = sum_k a_k exp(-((x-cx)^2 + (y-cy)^2) / (2 s^2)) + U[0, floor].
template <typename T>
__global__ void k_synth_latent(const double* blobs, int nblobs, int c, int h, int w,
                               double floor_amp, uint64_t seed, T* out) {
  const int fc = blockIdx.z;
  const double* B = blobs + (int64_t)fc * nblobs * 4;
  const int y = blockIdx.y, x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= w) return;
  // in the frame precision, like the blur
  T v = 0;
  for (int k = 0; k < nblobs; ++k) {
    const T a = (T)B[4 * k], s = (T)B[4 * k + 1], cx = (T)B[4 * k + 2], cy = (T)B[4 * k + 3];
    const T dx = (T)x - cx, dy = (T)y - cy;
    v += a * exp(-(dx * dx + dy * dy) / ((T)2 * s * s));
  }
  const int64_t oi = ((int64_t)fc * h + y) * w + x;
  v += (T)(floor_amp * uniform_at(seed, (uint64_t)oi, 2u));
  out[oi] = v;
}

// Multi-level security (Section 3): the private stream at a lower clearance
// level, its least significant bits removed.  code = rint(x (2^bits - 1))
// clamped to [0, 2^bits - 1], the `drop` low bits cleared, value
// code / (2^bits - 1); in double precision whatever the element type.
template <typename T>
__global__ void k_truncate_lsb(const T* in, int64_t count, int bits, int drop, T* out) {
  const double top = (double)((1ll << bits) - 1);
  const long long mask = ~((1ll << drop) - 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double c = fmin(fmax(rint((double)in[i] * top), 0.0), top);
    const long long code = (long long)c & mask;
    out[i] = (T)((double)code / top);
  }
}

// Camera side (Section 3, "Blur Kernel Selection": new random kernels for
// every frame): kernel `kind` of frame frame0 + f at redraw attempt[f],
// entries (Philox word + 1) 2^-32, uniform in (0, 1], normalised to unit sum
// in entry order.  Entry e is word e mod 4 of Philox(counter = (e / 4, frame,
// kind * 256 + attempt, 0), key = seed).  One thread per kernel; pairs whose
// active flag is clear keep their kernels.
__global__ void k_draw_kernels(int n, int t, int kind, int frame0, uint64_t seed, const int* active,
                               const int* attempt, double* kd) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n || !active[f]) return;
  double* K = kd + (int64_t)f * t * t;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int nn = t * t;
  double sum = 0.0;
  for (int b = 0; 4 * b < nn; ++b) {
    const U4 r = philox4x32_10({(uint32_t)b, (uint32_t)(frame0 + f), (uint32_t)(kind * 256 + attempt[f]), 0u},
                               k0, k1);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    for (int i = 0; i < 4 && 4 * b + i < nn; ++i) {
      const double u = u01(w[i]);
      K[4 * b + i] = u;
      sum += u;
    }
  }
  for (int e = 0; e < nn; ++e) K[e] = K[e] / sum;
}

}  // namespace

void launch_draw_kernels(int n, int t, int kind, int frame0, uint64_t seed, const int* active,
                         const int* attempt, double* kd, cudaStream_t st) {
  k_draw_kernels<<<(n + 127) / 128, 128, 0, st>>>(n, t, kind, frame0, seed, active, attempt, kd);
}

void launch_truncate_lsb(const void* in, int f64, int64_t count, int bits, int drop, void* out,
                         cudaStream_t st) {
  const int64_t blocks64 = (count + 255) / 256;
  const int blocks = (int)(blocks64 < 152 * 32 ? (blocks64 > 0 ? blocks64 : 1) : 152 * 32);
  if (f64) k_truncate_lsb<double><<<blocks, 256, 0, st>>>((const double*)in, count, bits, drop, (double*)out);
  else k_truncate_lsb<float><<<blocks, 256, 0, st>>>((const float*)in, count, bits, drop, (float*)out);
}

void launch_forward_blur(const void* latent, int n, int c, int h, int w, int f64,
                         const double* kernel, int t, double sigma, uint64_t seed, void* out,
                         cudaStream_t st) {
  const int hb = h + t - 1, wb = w + t - 1;
  dim3 g((wb + kTile - 1) / kTile, (hb + kTile - 1) / kTile, n * c);
  const int th = kTile + t - 1;
  const size_t sm = ((t * t * sizeof(double) + 15) & ~size_t(15)) + (size_t)th * th * (f64 ? 8 : 4);
  if (f64) {
    cudaFuncSetAttribute(k_forward_blur<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_forward_blur<double><<<g, kTile * 8, sm, st>>>((const double*)latent, c, h, w, kernel, t,
                                                      sigma, seed, (double*)out);
  } else if (t <= 17) {
    const float* L = (const float*)latent;
    float* o = (float*)out;
    switch (t) {
#define CBP_BLUR_CASE(T) \
  case T: launch_blur_rb<T>(L, n, c, h, w, kernel, sigma, seed, o, st); break;
      CBP_BLUR_CASE(1) CBP_BLUR_CASE(2) CBP_BLUR_CASE(3) CBP_BLUR_CASE(4) CBP_BLUR_CASE(5)
      CBP_BLUR_CASE(6) CBP_BLUR_CASE(7) CBP_BLUR_CASE(8) CBP_BLUR_CASE(9) CBP_BLUR_CASE(10)
      CBP_BLUR_CASE(11) CBP_BLUR_CASE(12) CBP_BLUR_CASE(13) CBP_BLUR_CASE(14) CBP_BLUR_CASE(15)
      CBP_BLUR_CASE(16) default: CBP_BLUR_CASE(17)
#undef CBP_BLUR_CASE
    }
  } else {
    cudaFuncSetAttribute(k_forward_blur<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_forward_blur<float><<<g, kTile * 8, sm, st>>>((const float*)latent, c, h, w, kernel, t,
                                                     sigma, seed, (float*)out);
  }
}

void launch_synth_latent(const double* blobs, int nblobs, int n, int c, int h, int w, int f64,
                         double floor_amp, uint64_t seed, void* out, cudaStream_t st) {
  dim3 g((w + 127) / 128, h, n * c);
  if (f64)
    k_synth_latent<double><<<g, 128, 0, st>>>(blobs, nblobs, c, h, w, floor_amp, seed, (double*)out);
  else
    k_synth_latent<float><<<g, 128, 0, st>>>(blobs, nblobs, c, h, w, floor_amp, seed, (float*)out);
}

}  // namespace cbp
