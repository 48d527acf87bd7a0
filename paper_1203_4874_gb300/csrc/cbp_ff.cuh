// Float-float arithmetic on the single-precision units: a value hi + lo with
// |lo| <= ulp(hi) / 2, about 48 significant bits (Dekker 1971; Knuth's
// two-sum and the FMA-based exact product).  On this GPU a double-precision
// instruction occupies a scheduler's double unit for about 64 cycles against
// one cycle for a single-precision one, so sums and products of a few dozen
// terms that need ~1e-14 relative accuracy run several times faster here.
#pragma once
#include "cbp_common.cuh"

namespace cbp {

struct fx {
  float hi, lo;
};

// exact a + b = s + e
__device__ __forceinline__ fx fx_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// renormalise s + e with |e| small against s
__device__ __forceinline__ fx fx_norm(float s, float e) {
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ fx fx_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double fx_val(fx a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ fx fx_add(fx a, fx b) {
  const fx s = fx_two_sum(a.hi, b.hi);
  return fx_norm(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ fx fx_neg(fx a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ fx fx_mul(fx a, fx b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fx_norm(p, e);
}
__device__ __forceinline__ fx fx_scale(fx a, float s) {   // a * s, s a single-precision value
  const float p = a.hi * s;
  return fx_norm(p, fmaf(a.hi, s, -p) + a.lo * s);
}
__device__ __forceinline__ fx fx_sub(fx a, fx b) { return fx_add(a, fx_neg(b)); }
// a / b: a single-precision quotient, corrected once by the exactly formed
// remainder a - q b (long division with two digits)
__device__ __forceinline__ fx fx_div(fx a, fx b) {
  const float q1 = __fdividef(a.hi, b.hi);
  const float p = q1 * b.hi;
  const float pe = fmaf(q1, b.hi, -p);                      // q1 b.hi = p + pe exactly
  const float r = (((a.hi - p) - pe) + a.lo) - q1 * b.lo;   // a - q1 b
  return fx_norm(q1, __fdividef(r, b.hi));
}
__device__ __forceinline__ fx fx_ldexp(fx a, int e) { return {ldexpf(a.hi, e), ldexpf(a.lo, e)}; }
__device__ __forceinline__ float fx_abs_hi(fx a) { return fabsf(a.hi); }
__device__ __forceinline__ bool fx_neg_sign(fx a) { return a.hi < 0.f || (a.hi == 0.f && a.lo < 0.f); }
__device__ __forceinline__ bool fx_is_zero(fx a) { return a.hi == 0.f && a.lo == 0.f; }

// Accumulator for sums of products: the products' high parts are added by
// two-sum, every rounding term gathered in lo without renormalising (a few
// dozen terms keep lo within ~1e-14 of the sum's magnitude); value() at the end.
struct fx_acc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(fx b) {
    const fx s = fx_two_sum(hi, b.hi);
    hi = s.hi;
    lo += s.lo + b.lo;
  }
  __device__ __forceinline__ void mac(fx a, fx b) {   // += a b
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
    const fx s = fx_two_sum(hi, p);
    hi = s.hi;
    lo += s.lo + e;
  }
  __device__ __forceinline__ fx value() const { return fx_norm(hi, lo); }
};

// complex float-float
struct cfx {
  fx re, im;
};
__device__ __forceinline__ cfx cfx_of(cd a) { return {fx_of(a.re), fx_of(a.im)}; }
__device__ __forceinline__ cd cfx_val(cfx a) { return mk(fx_val(a.re), fx_val(a.im)); }
struct cfx_acc {
  fx_acc re, im;
  __device__ __forceinline__ void mac(cfx a, cfx b) {   // += a b
    re.mac(a.re, b.re);
    re.mac(fx_neg(a.im), b.im);
    im.mac(a.re, b.im);
    im.mac(a.im, b.re);
  }
  __device__ __forceinline__ void macc(cfx a, cfx b) {  // += conj(a) b
    re.mac(a.re, b.re);
    re.mac(a.im, b.im);
    im.mac(a.re, b.im);
    im.mac(fx_neg(a.im), b.re);
  }
  __device__ __forceinline__ cfx value() const { return {re.value(), im.value()}; }
};
__device__ __forceinline__ cfx cfx_mul(cfx a, cfx b) {
  cfx_acc s;
  s.mac(a, b);
  return s.value();
}

}  // namespace cbp
