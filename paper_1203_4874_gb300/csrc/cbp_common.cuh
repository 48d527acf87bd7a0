// Shared device helpers of libcbp: complex arithmetic, reductions, launch checks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

namespace cbp {

template <typename T> struct alignas(2 * sizeof(T)) cpx { T re, im; };
using cf = cpx<float>;
using cd = cpx<double>;

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T r, T i) { return {r, i}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> operator*(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> conj(cpx<T> a) { return {a.re, -a.im}; }
template <typename T> __host__ __device__ __forceinline__ T abs2(cpx<T> a) { return a.re * a.re + a.im * a.im; }
// conj(a) * b
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc += a * b
template <typename T> __host__ __device__ __forceinline__ void cfma(cpx<T>& acc, cpx<T> a, cpx<T> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += conj(a) * b
template <typename T> __host__ __device__ __forceinline__ void cfmac(cpx<T>& acc, cpx<T> a, cpx<T> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
template <typename D, typename S> __host__ __device__ __forceinline__ cpx<D> cvt(cpx<S> a) {
  return {(D)a.re, (D)a.im};
}

// A complex double held as two float-float numbers (hi + lo each), for
// extended-precision arithmetic on the single-precision units.
struct alignas(16) cdf { float rh, rl, ih, il; };
__host__ __device__ __forceinline__ cdf to_cdf(cd a) {
  const float rh = (float)a.re, ih = (float)a.im;
  return {rh, (float)(a.re - (double)rh), ih, (float)(a.im - (double)ih)};
}

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
  __device__ __forceinline__ void merge(const TwoSum& o) {
    add(o.hi);
    lo += o.lo;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  __device__ __forceinline__ bool finite() const { return isfinite(hi) && isfinite(lo); }
  // 8-byte bin: (hi, lo) as two floats
  __device__ __forceinline__ void store(void* p) const { *(float2*)p = make_float2(hi, lo); }
};
struct DoubleSum {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void merge(const DoubleSum& o) { v += o.v; }
  __device__ __forceinline__ double value() const { return v; }
  __device__ __forceinline__ bool finite() const { return isfinite(v); }
  __device__ __forceinline__ void store(void* p) const { *(double*)p = v; }
};

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <typename T> __device__ __forceinline__ T ld_elem(const void* p, int64_t i) {
  return (T)(((const T*)p)[i]);
}

// Base address of frame f of a batch: from the table if present, else strided.
template <class FD> __device__ __forceinline__ const void* frame_base(const FD& fr, int f) {
  if (fr.tab) return (const void*)fr.tab[f];
  return (const char*)fr.data + (size_t)f * (size_t)fr.fs * (fr.f64 ? 8u : 4u);
}

// Load one element of a frame batch stored as float or double, converted to T.
template <typename T> __device__ __forceinline__ T ld_frame(const void* p, int64_t i, int is_f64) {
  return is_f64 ? (T)__ldg(((const double*)p) + i) : (T)__ldg(((const float*)p) + i);
}

// Bounds-checked builds (-DCBP_CHECKS).  CBP_CHECK(cond, site) guards one
// access: in a normal build it is `true` and costs nothing; in a checked
// build a failed condition sets bit `site` (0..31) of this source file's
// check word and yields false, so the caller skips the access instead of
// faulting.  CBP_CHECKS_TU(id) (once per source file) makes the file's word
// readable through cbp_check_words() as word `id`.
void register_check_word(int id, unsigned (*read)(bool reset));
#ifdef CBP_CHECKS
static __device__ unsigned cbp_check_word;
__device__ __forceinline__ bool cbp_check(bool ok, int site) {
  if (!ok) atomicOr(&cbp_check_word, 1u << (site & 31));
  return ok;
}
#define CBP_CHECK(cond, site) (::cbp::cbp_check((cond), (site)))
#define CBP_CHECKS_TU(id)                                                     \
  static unsigned cbp_read_check_word(bool reset) {                         \
    unsigned v = 0;                                                         \
    cudaMemcpyFromSymbol(&v, cbp_check_word, sizeof v);                     \
    if (reset) {                                                            \
      const unsigned z = 0;                                                 \
      cudaMemcpyToSymbol(cbp_check_word, &z, sizeof z);                     \
    }                                                                       \
    return v;                                                               \
  }                                                                         \
  static const bool cbp_check_word_registered =                             \
      (::cbp::register_check_word((id), cbp_read_check_word), true);
#else
#define CBP_CHECK(cond, site) (true)
#define CBP_CHECKS_TU(id)
#endif
// Check-word numbers of the source files.
enum CheckTu { kChkFft = 0, kChkColpass, kChkEval, kChkSolve, kChkCnn, kChkForward, kChkWords };

}  // namespace cbp
