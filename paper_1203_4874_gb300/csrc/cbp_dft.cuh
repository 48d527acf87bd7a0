// In-register DFTs of small sizes (the butterflies of the library's FFTs) and
// compile-time twiddle constants.
#pragma once
#include "cbp_common.cuh"

namespace cbp {

// Butterfly arithmetic: complex add and subtract, and a real multiple of a
// complex value, alone or added to another.  For float data on this GPU each
// is one paired FP32 instruction on a (re, im) register pair, rounded exactly
// like the two scalar operations it replaces (a - b as the fused b * -1 + a;
// s a + c fused, as the scalar code contracts it).  -DCBP_F32X2=0 keeps them
// scalar.
#ifndef CBP_F32X2
#define CBP_F32X2 1
#endif
template <typename T> __device__ __forceinline__ cpx<T> bf_add(cpx<T> a, cpx<T> b) { return a + b; }
template <typename T> __device__ __forceinline__ cpx<T> bf_sub(cpx<T> a, cpx<T> b) { return a - b; }
template <typename T> __device__ __forceinline__ cpx<T> bf_scale(T s, cpx<T> a) { return s * a; }
template <typename T> __device__ __forceinline__ cpx<T> bf_fma(T s, cpx<T> a, cpx<T> c) {
  return mk<T>(fma(s, a.re, c.re), fma(s, a.im, c.im));
}
#if CBP_F32X2 && defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000)
__device__ __forceinline__ float2 bf_f2(cf a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ cf bf_cf(float2 a) { return mk(a.x, a.y); }
template <> __device__ __forceinline__ cf bf_add<float>(cf a, cf b) { return bf_cf(__fadd2_rn(bf_f2(a), bf_f2(b))); }
template <> __device__ __forceinline__ cf bf_sub<float>(cf a, cf b) {
  return bf_cf(__ffma2_rn(bf_f2(b), make_float2(-1.f, -1.f), bf_f2(a)));
}
template <> __device__ __forceinline__ cf bf_scale<float>(float s, cf a) {
  return bf_cf(__fmul2_rn(make_float2(s, s), bf_f2(a)));
}
template <> __device__ __forceinline__ cf bf_fma<float>(float s, cf a, cf c) {
  return bf_cf(__ffma2_rn(make_float2(s, s), bf_f2(a), bf_f2(c)));
}
#endif

// In-register DFTs of size R (Inv: e^{+i...}, unnormalised), float constants
// for float data.  Radix 8 = 2 x 4 and radix 9 = 3 x 3 with internal twiddles.
// Products by +-i stay scalar (a swap and a sign, free in scalar adds).
template <typename T, bool Inv>
__device__ __forceinline__ cpx<T> mul_i(cpx<T> d) {     // (Inv ? +i : -i) * d
  return Inv ? mk<T>(-d.im, d.re) : mk<T>(d.im, -d.re);
}

template <typename T, bool Inv>
__device__ __forceinline__ void dft2(cpx<T>& a, cpx<T>& b) {
  const cpx<T> t = bf_sub(a, b);
  a = bf_add(a, b);
  b = t;
}

template <typename T, bool Inv>
__device__ __forceinline__ void dft3(cpx<T>& a, cpx<T>& b, cpx<T>& c) {
  const T h = (T)0.86602540378443864676;       // sin(2 pi / 3)
  const cpx<T> sm = bf_add(b, c), d = bf_sub(b, c);
  const cpx<T> t1 = bf_fma((T)-0.5, sm, a);
  const cpx<T> t2 = h * mul_i<T, Inv>(d);
  a = bf_add(a, sm);
  b = bf_add(t1, t2);
  c = bf_sub(t1, t2);
}

template <typename T, bool Inv>
__device__ __forceinline__ void dft4(cpx<T>& v0, cpx<T>& v1, cpx<T>& v2, cpx<T>& v3) {
  const cpx<T> t0 = bf_add(v0, v2), t1 = bf_sub(v0, v2), t2 = bf_add(v1, v3);
  const cpx<T> t3 = mul_i<T, Inv>(bf_sub(v1, v3));
  v0 = bf_add(t0, t2);
  v2 = bf_sub(t0, t2);
  v1 = t1 + t3;
  v3 = t1 - t3;
}

// odd prime radix by symmetric pairs; C, S = cos, sin(2 pi j / R)
template <typename T, bool Inv, int R>
__device__ __forceinline__ void dft_odd(cpx<T>* v, const T* C, const T* S) {
  constexpr int H = (R - 1) / 2;
  cpx<T> a[H], b[H];
#pragma unroll
  for (int m = 1; m <= H; ++m) {
    a[m - 1] = bf_add(v[m], v[R - m]);
    b[m - 1] = bf_sub(v[m], v[R - m]);
  }
  const cpx<T> x0 = v[0];
  cpx<T> s0 = x0;
#pragma unroll
  for (int m = 0; m < H; ++m) s0 = bf_add(s0, a[m]);
  v[0] = s0;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    cpx<T> re = x0, im = mk<T>(0, 0);
#pragma unroll
    for (int m = 1; m <= H; ++m) {
      const int j = (k * m) % R;
      re = bf_fma(C[j], a[m - 1], re);
      im = bf_fma(S[j], b[m - 1], im);
    }
    const cpx<T> si = mul_i<T, Inv>(im);   // forward: X[k] = re - i im, X[R-k] = re + i im
    v[k] = re + si;
    v[R - k] = re - si;
  }
}

template <typename T, bool Inv, int R>
__device__ __forceinline__ void small_dft(cpx<T>* v) {
  if constexpr (R == 2) {
    dft2<T, Inv>(v[0], v[1]);
  } else if constexpr (R == 3) {
    dft3<T, Inv>(v[0], v[1], v[2]);
  } else if constexpr (R == 4) {
    dft4<T, Inv>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 5) {
    const T C[5] = {(T)1, (T)0.30901699437494742410, (T)-0.80901699437494742410,
                    (T)-0.80901699437494742410, (T)0.30901699437494742410};
    const T S[5] = {(T)0, (T)0.95105651629515357212, (T)0.58778525229247312917,
                    (T)-0.58778525229247312917, (T)-0.95105651629515357212};
    dft_odd<T, Inv, 5>(v, C, S);
  } else if constexpr (R == 7) {
    const T C[7] = {(T)1, (T)0.62348980185873353053, (T)-0.22252093395631440429,
                    (T)-0.90096886790241912624, (T)-0.90096886790241912624,
                    (T)-0.22252093395631440429, (T)0.62348980185873353053};
    const T S[7] = {(T)0, (T)0.78183148246802980871, (T)0.97492791218182360702,
                    (T)0.43388373911755812048, (T)-0.43388373911755812048,
                    (T)-0.97492791218182360702, (T)-0.78183148246802980871};
    dft_odd<T, Inv, 7>(v, C, S);
  } else if constexpr (R == 8) {
    // even / odd halves by radix 4, combined with w8^k
    dft4<T, Inv>(v[0], v[2], v[4], v[6]);
    dft4<T, Inv>(v[1], v[3], v[5], v[7]);
    const T r = (T)0.70710678118654752440;
    const cpx<T> o1 = bf_scale(r, v[3] + mul_i<T, Inv>(v[3]));     // w8^1 = r (1 -/+ i)
    const cpx<T> o2 = mul_i<T, Inv>(v[5]);                          // w8^2 = -/+ i
    const cpx<T> o3 = bf_scale(r, mul_i<T, Inv>(v[7]) - v[7]);     // w8^3 = r (-1 -/+ i)
    const cpx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    v[0] = bf_add(e0, v[1]);
    v[4] = bf_sub(e0, v[1]);
    v[1] = bf_add(e1, o1);
    v[5] = bf_sub(e1, o1);
    v[2] = e2 + o2;
    v[6] = e2 - o2;
    v[3] = bf_add(e3, o3);
    v[7] = bf_sub(e3, o3);
  } else {  // R == 9: 3 x 3
    dft3<T, Inv>(v[0], v[3], v[6]);
    dft3<T, Inv>(v[1], v[4], v[7]);
    dft3<T, Inv>(v[2], v[5], v[8]);
    // twiddles w9^{n2 k1}: (n2, k1) = (1,1) (1,2) (2,1) (2,2) -> w9^1, w9^2, w9^2, w9^4
    const T c1 = (T)0.76604444311897803520, s1 = (T)0.64278760968653932632;   // 2 pi / 9
    const T c2 = (T)0.17364817766693034885, s2 = (T)0.98480775301220805936;   // 4 pi / 9
    const T c4 = (T)-0.93969262078590838405, s4 = (T)0.34202014332566873304;  // 8 pi / 9
    const T sg = Inv ? (T)1 : (T)-1;
    v[4] = v[4] * mk<T>(c1, sg * s1);
    v[7] = v[7] * mk<T>(c2, sg * s2);
    v[5] = v[5] * mk<T>(c2, sg * s2);
    v[8] = v[8] * mk<T>(c4, sg * s4);
    // v[n2 + 3 k1] holds Y_{n2}[k1]; DFT3 over n2 for each k1 -> X[k1 + 3 k2]
    cpx<T> a0 = v[0], a1 = v[1], a2 = v[2];
    dft3<T, Inv>(a0, a1, a2);
    cpx<T> b0 = v[3], b1 = v[4], b2 = v[5];
    dft3<T, Inv>(b0, b1, b2);
    cpx<T> d0 = v[6], d1 = v[7], d2 = v[8];
    dft3<T, Inv>(d0, d1, d2);
    v[0] = a0; v[3] = a1; v[6] = a2;
    v[1] = b0; v[4] = b1; v[7] = b2;
    v[2] = d0; v[5] = d1; v[8] = d2;
  }
}

// ------------------------------------------------ compile-time twiddles ---
// cos and sin of 2 pi m / n for integers m, n, evaluated by the compiler: the
// angle is reduced to an octant exactly in integer arithmetic, then Taylor
// series on [0, pi/4] (terms to x^27: below double rounding there).
constexpr double kTwoPi = 6.283185307179586476925286766559;

constexpr double cx_taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / (double)((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
constexpr double cx_taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x * x / (double)((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}
// (cos, sin) of 2 pi m / n
struct CxCS {
  double c, s;
};
constexpr CxCS cx_cossin(long long m, long long n) {
  m %= n;
  if (m < 0) m += n;
  // octant o = floor(8 m / n); remainder angle r = 2 pi (m / n - o / 8) in [0, pi/4)
  const long long o = (8 * m) / n;
  const double r = kTwoPi * (double)(8 * m - o * n) / (double)(8 * n);
  const double cr = cx_taylor_cos(r), sr = cx_taylor_sin(r);
  const double h = 0.70710678118654752440;   // cos(pi/4) = sin(pi/4)
  // angle = o pi/4 + r
  switch (o) {
    case 0: return {cr, sr};
    case 1: return {h * (cr - sr), h * (cr + sr)};
    case 2: return {-sr, cr};
    case 3: return {-h * (cr + sr), h * (cr - sr)};
    case 4: return {-cr, -sr};
    case 5: return {-h * (cr - sr), -h * (cr + sr)};
    case 6: return {sr, -cr};
    default: return {h * (cr + sr), -h * (cr - sr)};
  }
}

// Table of w_N^k = exp(-2 pi i k / N), k < N, in single precision.
template <int N>
struct TwTable {
  float re[N], im[N];
  constexpr TwTable() : re(), im() {
    for (int k = 0; k < N; ++k) {
      const CxCS v = cx_cossin(k, N);
      re[k] = (float)v.c;
      im[k] = (float)-v.s;
    }
  }
};

// w_N^m (forward sign; Inv: conjugate) from a compile-time table: with m a
// constant after unrolling, both parts are immediates.
template <int N, bool Inv>
__device__ __forceinline__ cf tw_const(int m) {
  constexpr TwTable<N> t{};
  const int k = m % N;
  return mk(t.re[k], Inv ? -t.im[k] : t.im[k]);
}

// ------------------------------------------------- composite DFTs in registers
// DFT of N = A B points held by one thread, in place: element n = a + A b on
// input.  B-point DFTs over b for each a, the twiddles w_N^(a kb), then A-point
// DFTs over a for each kb; X[kb + B ka] ends up in v[ka + A kb] (dft_pos).
template <int A, int B>
__host__ __device__ constexpr int dft_pos(int k) {
  return (k / B) + A * (k % B);
}

template <bool Inv, int A, int B>
__device__ __forceinline__ void dft_ab(cf* v) {
  constexpr int N = A * B;
#pragma unroll
  for (int a = 0; a < A; ++a) {
    cf t[B];
#pragma unroll
    for (int b = 0; b < B; ++b) t[b] = v[a + A * b];
    small_dft<float, Inv, B>(t);
#pragma unroll
    for (int kb = 0; kb < B; ++kb) v[a + A * kb] = (a * kb) % N ? t[kb] * tw_const<N, Inv>(a * kb) : t[kb];
  }
#pragma unroll
  for (int kb = 0; kb < B; ++kb) {
    cf t[A];
#pragma unroll
    for (int a = 0; a < A; ++a) t[a] = v[a + A * kb];
    small_dft<float, Inv, A>(t);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) v[ka + A * kb] = t[ka];
  }
}

// The composite sizes of the fused column pass.
template <int N> struct RegDft;
template <> struct RegDft<32> { static constexpr int A = 4, B = 8; };
template <> struct RegDft<35> { static constexpr int A = 5, B = 7; };
template <> struct RegDft<36> { static constexpr int A = 4, B = 9; };
template <> struct RegDft<27> { static constexpr int A = 3, B = 9; };

// v[0..N) natural order in, X[k] at v[reg_pos<N>(k)] out.
template <bool Inv, int N>
__device__ __forceinline__ void reg_dft(cf* v) {
  dft_ab<Inv, RegDft<N>::A, RegDft<N>::B>(v);
}
template <int N>
__host__ __device__ constexpr int reg_pos(int k) {
  return dft_pos<RegDft<N>::A, RegDft<N>::B>(k);
}

}  // namespace cbp
