// Smallest eigenpair of a Hermitian (or real symmetric) n x n matrix by one
// warp, n <= 64: the null vector of the per-sample normal matrix G = S^H S
// (Eq. 4; Section 5 takes it from an SVD of the Bezout/Sylvester matrix).
//
//   1. Householder reduction to a real symmetric tridiagonal T = Q^H G Q
//      (reflectors H_k = I - tau_k v_k v_k^H chosen so that beta_k is real);
//   2. Sturm counts by multisection (each lane counts at its own shift) for
//      the two smallest and the largest eigenvalue of T: single-precision
//      rounds down to the single-precision floor, then double-precision
//      rounds inside the widened brackets;
//   3. inverse iteration on T - sigma I (tridiagonal LU with row interchanges)
//      with sigma inside the bracket of the smallest eigenvalue;
//   4. x = Q y;
//   5. optional Newton steps against an exact operator (S^H S applied through
//      S): the correction equation (G - theta) d = -r, d orthogonal to x, is
//      solved through T in Olsen's form d = -(G - theta)^{-1} r +
//      eps (G - theta)^{-1} x.
//
// Every step is O(n^2) per lane-column except the reduction (O(n^3) in all),
// and all but the first bisection rounds run in double precision: a GPU whose
// double pipe is narrow spends its time on the reduction's rank-2 updates,
// n^3 / 3 complex multiply-adds in all.  Sign and exponent tests use the
// integer pipe; reciprocals start from a single-precision seed.
//
// Lane l owns the columns l and l + 32.  The matrix is stored in full with row
// stride n; lane i touches element (j, i) of row j, so every access of a row
// is contiguous across the warp.  Included inside namespace cbp::(anonymous)
// of the solver's translation unit, after its scalar helpers (fma_, to_cd,
// re_, cj_, a2_, Ops).

__device__ __forceinline__ double im_(double) { return 0.0; }
__device__ __forceinline__ float im_(float) { return 0.f; }
template <typename T> __device__ __forceinline__ T im_(cpx<T> x) { return x.im; }
template <typename E, typename R> __device__ __forceinline__ E mk_e(R re, R im);
template <> __device__ __forceinline__ double mk_e<double, double>(double re, double) { return re; }
template <> __device__ __forceinline__ cd mk_e<cd, double>(double re, double im) { return mk(re, im); }
template <> __device__ __forceinline__ cf mk_e<cf, float>(float re, float im) { return mk(re, im); }
__device__ __forceinline__ double mul_(double a, double b) { return a * b; }
template <typename T> __device__ __forceinline__ cpx<T> mul_(cpx<T> a, cpx<T> b) { return a * b; }
__device__ __forceinline__ double sc_(double s, double a) { return s * a; }
template <typename T> __device__ __forceinline__ cpx<T> sc_(T s, cpx<T> a) { return s * a; }
__device__ __forceinline__ void fma_(cf& acc, cf a, cf b) { cfma(acc, a, b); }
__device__ __forceinline__ cf warp_sum_e(cf v) { return mk(warp_sum(v.re), warp_sum(v.im)); }
// real scalar type of an element type
template <typename E> struct RealOf { using type = E; };
template <typename T> struct RealOf<cpx<T>> { using type = T; };
// reflector element -> vector element
__device__ __forceinline__ cd to_v(double x, cd) { return mk(x, 0.0); }
__device__ __forceinline__ cd to_v(cd x, cd) { return x; }
__device__ __forceinline__ cf to_v(cf x, cf) { return x; }

// Per-warp work area.
struct TriWs {
  void* A;        // E[n * n]: the matrix; row k then holds reflector v_k (k+1..n-1); 16 (n^2 + n)
                  // bytes: the single-precision path keeps Q (cf [n][n + 1]) behind its reflectors
  void* tau;      // E[n]
  void* w;        // E[n]
  double* d;      // [n] diagonal of T
  double* e;      // [n] off-diagonal of T: e[k] couples rows k and k + 1
  double* e2;     // [n] e^2
  double* u0;     // [n] LU of T - sigma I: diagonal of U
  double* u1;     // [n] first superdiagonal of U
  double* u2;     // [n] second superdiagonal of U (row interchanges)
  double* lm;     // [n] multipliers
  int* piv;       // [n] 1 where rows k and k + 1 were interchanged
  float* df;      // [n] d in single precision
  float* e2f;     // [n] e^2 in single precision
  int* iv;        // [4] values broadcast to the CTA
  void* part;     // [8][n] complex: per-warp partial sums of the CTA's reduction
  cd* x;          // [n] the eigenvector of G
  cd* r;          // [n] residual
  cd* z;          // [n] scratch (T coordinates)
  cd* q;          // [n] scratch (T coordinates)
};

// Bytes of one warp's work area; a multiple of 128, so that every warp's area
// (placed back to back) and each of its 16-byte-aligned parts stay aligned.
__host__ __device__ inline size_t tri_ws_bytes(int n) {
  const size_t b = (size_t)16 * ((size_t)n * n + 3 * n) + (size_t)8 * 7 * n + (size_t)4 * 3 * n +
                   16 + (size_t)16 * 4 * n + (size_t)16 * 8 * n + 16 * 19;   // + alignment of the 19 parts
  return (b + 127) & ~size_t(127);
}

__device__ inline TriWs carve_tri(char* p, int n) {
  TriWs W;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += (bytes + 15) & ~size_t(15);
    return q;
  };
  W.A = take((size_t)16 * n * n + (size_t)16 * n);
  W.tau = take((size_t)16 * n);
  W.w = take((size_t)16 * n);
  W.x = (cd*)take((size_t)16 * n);
  W.r = (cd*)take((size_t)16 * n);
  W.z = (cd*)take((size_t)16 * n);
  W.q = (cd*)take((size_t)16 * n);
  W.d = (double*)take((size_t)8 * n);
  W.e = (double*)take((size_t)8 * n);
  W.e2 = (double*)take((size_t)8 * n);
  W.u0 = (double*)take((size_t)8 * n);
  W.u1 = (double*)take((size_t)8 * n);
  W.u2 = (double*)take((size_t)8 * n);
  W.lm = (double*)take((size_t)8 * n);
  W.piv = (int*)take((size_t)4 * n);
  W.df = (float*)take((size_t)4 * n);
  W.e2f = (float*)take((size_t)4 * n);
  W.iv = (int*)take(16);
  W.part = take((size_t)16 * 8 * n);
  return W;
}

// 1. Householder reduction.  On return T = (d, e), tau and the reflectors
// (row k of A from column k + 1 on, v_k[k + 1] = 1) describe
// Q = H_0 H_1 ... H_{n-2} with A_in = Q T Q^H.
template <typename E>
__device__ void tri_reduce(E* A, E* tau, E* w, typename RealOf<E>::type* d,
                           typename RealOf<E>::type* e, int n) {
  using R = typename RealOf<E>::type;
  const int lane = threadIdx.x & 31;
  for (int k = 0; k + 1 < n; ++k) {
    const int k1 = k + 1;
    E* vk = A + (size_t)k * n;             // row k = conj(column k)
    const E alpha = cj_(vk[k1]);
    R xn2 = R(0);
    for (int i = lane; i < n; i += 32)
      if (i > k1) xn2 += a2_(vk[i]);
    xn2 = warp_sum(xn2);
    const R ar = re_(alpha), ai = im_(alpha);
    E tk = Ops<E>::z();
    R beta = ar;
    if (xn2 > R(0) || ai != R(0)) {
      // H^H (alpha, x) = (beta, 0) with beta real, |beta| = |(alpha, x)|
      beta = -copysign(sqrt(ar * ar + ai * ai + xn2), ar);
      const R ib = R(1) / beta;
      tk = mk_e<E, R>((beta - ar) * ib, -ai * ib);
      // v = x / (alpha - beta)
      const R dr = ar - beta, dn = R(1) / (dr * dr + ai * ai);
      const E scl = mk_e<E, R>(dr * dn, -ai * dn);
      __syncwarp();
      for (int i = lane; i < n; i += 32) {
        if (i > k1) vk[i] = mul_(cj_(vk[i]), scl);
        else if (i == k1) vk[i] = Ops<E>::o();
      }
    } else {
      __syncwarp();
      for (int i = lane; i < n; i += 32)
        if (i == k1) vk[i] = Ops<E>::o();
    }
    if (lane == 0) {
      d[k] = re_(A[(size_t)k * n + k]);
      e[k] = beta;
      tau[k] = tk;
    }
    __syncwarp();
    if (!Ops<E>::nz(tk)) continue;
    // y = tau A v over the trailing block; w = y - (1/2) conj(tau) (v^H y) v
    E y[2];
    E dotl = Ops<E>::z();
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = lane + 32 * c;
      y[c] = Ops<E>::z();
      if (i > k && i < n) {
        E acc = Ops<E>::z(), acc1 = Ops<E>::z();   // two chains for latency
        int j = k1;
        for (; j + 1 < n; j += 2) {
          fma_(acc, cj_(A[(size_t)j * n + i]), vk[j]);
          fma_(acc1, cj_(A[(size_t)(j + 1) * n + i]), vk[j + 1]);
        }
        if (j < n) fma_(acc, cj_(A[(size_t)j * n + i]), vk[j]);
        acc = acc + acc1;
        y[c] = mul_(tk, acc);
        fma_(dotl, cj_(vk[i]), y[c]);
      }
    }
    const E dot = warp_sum_e(dotl);
    const R hc = R(0.5) * re_(mul_(cj_(tk), dot));
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = lane + 32 * c;
      if (i > k && i < n) {
        y[c] = y[c] - sc_(hc, vk[i]);
        w[i] = y[c];
      }
    }
    __syncwarp();
    // A <- A - v w^H - w v^H on the trailing block
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = lane + 32 * c;
      if (i > k && i < n) {
        const E cw = cj_(y[c]), cv = cj_(vk[i]);
        for (int j = k1; j < n; ++j) {
          E t = mul_(vk[j], cw);
          fma_(t, w[j], cv);
          A[(size_t)j * n + i] = A[(size_t)j * n + i] - t;
        }
      }
    }
    __syncwarp();
  }
  if (lane == 0) d[n - 1] = re_(A[(size_t)(n - 1) * n + n - 1]);
  __syncwarp();
}

// Sign and zero tests of a double on the integer pipe.
__device__ __forceinline__ bool dneg(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool dzero(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ int dexp(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// The same reduction by all warps of the CTA (real samples, whose solve has a
// CTA to itself): the lead warp forms each reflector; the matrix-vector
// product and the rank-2 update are split by rows j = w (mod warps), the
// product's per-warp partial sums meeting in part[w][i].
template <typename E>
__device__ void tri_reduce_block(E* A, E* tau, E* w, typename RealOf<E>::type* d,
                                 typename RealOf<E>::type* e, int n, E* part /* [8][n] */) {
  using R = typename RealOf<E>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = min(8, (int)(blockDim.x >> 5));   // warps taking part
  if (warp >= nw) {                                 // the others only keep the barriers
    for (int k = 0; k + 1 < n; ++k) {
      __syncthreads();
      if (!Ops<E>::nz(tau[k])) continue;
      __syncthreads();
      __syncthreads();
      __syncthreads();
    }
    __syncthreads();
    return;
  }
  for (int k = 0; k + 1 < n; ++k) {
    const int k1 = k + 1;
    E* vk = A + (size_t)k * n;
    if (warp == 0) {
      const E alpha = cj_(vk[k1]);
      R xn2 = R(0);
      for (int i = lane; i < n; i += 32)
        if (i > k1) xn2 += a2_(vk[i]);
      xn2 = warp_sum(xn2);
      const R ar = re_(alpha), ai = im_(alpha);
      E tk = Ops<E>::z();
      R beta = ar;
      if (xn2 > R(0) || ai != R(0)) {
        beta = -copysign(sqrt(ar * ar + ai * ai + xn2), ar);
        const R ib = R(1) / beta;
        tk = mk_e<E, R>((beta - ar) * ib, -ai * ib);
        const R dr = ar - beta, dn = R(1) / (dr * dr + ai * ai);
        const E scl = mk_e<E, R>(dr * dn, -ai * dn);
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
          if (i > k1) vk[i] = mul_(cj_(vk[i]), scl);
          else if (i == k1) vk[i] = Ops<E>::o();
        }
      } else {
        __syncwarp();
        for (int i = lane; i < n; i += 32)
          if (i == k1) vk[i] = Ops<E>::o();
      }
      if (lane == 0) {
        d[k] = re_(A[(size_t)k * n + k]);
        e[k] = beta;
        tau[k] = tk;
      }
    }
    __syncthreads();
    const E tk = tau[k];
    if (!Ops<E>::nz(tk)) continue;
    // partial products over this warp's rows
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = lane + 32 * c;
      if (i > k && i < n) {
        E acc = Ops<E>::z();
        for (int j = k1 + warp; j < n; j += nw) fma_(acc, cj_(A[(size_t)j * n + i]), vk[j]);
        part[warp * n + i] = acc;
      }
    }
    __syncthreads();
    if (warp == 0) {
      E y[2];
      E dotl = Ops<E>::z();
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int i = lane + 32 * c;
        y[c] = Ops<E>::z();
        if (i > k && i < n) {
          E acc = part[i];
          for (int ww = 1; ww < nw; ++ww) acc = acc + part[ww * n + i];
          y[c] = mul_(tk, acc);
          fma_(dotl, cj_(vk[i]), y[c]);
        }
      }
      const E dot = warp_sum_e(dotl);
      const R hc = R(0.5) * re_(mul_(cj_(tk), dot));
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int i = lane + 32 * c;
        if (i > k && i < n) w[i] = y[c] - sc_(hc, vk[i]);
      }
    }
    __syncthreads();
    // rank-2 update of this warp's rows
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = lane + 32 * c;
      if (i > k && i < n) {
        const E cw = cj_(w[i]), cv = cj_(vk[i]);
        for (int j = k1 + warp; j < n; j += nw) {
          E t = mul_(vk[j], cw);
          fma_(t, w[j], cv);
          A[(size_t)j * n + i] = A[(size_t)j * n + i] - t;
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) d[n - 1] = re_(A[(size_t)(n - 1) * n + n - 1]);
  __syncthreads();
}

// Number of eigenvalues of T below sig: sign changes of the leading principal
// minors p_i = det(T_i - sig I) (p_i = (d_i - sig) p_{i-1} - e_{i-1}^2 p_{i-2};
// a zero minor takes the sign opposite to its predecessor's).  The minors
// are rescaled by powers of two when they leave [2^-600, 2^600].
__device__ __forceinline__ int sturm_count(const double* d, const double* e2, int n, double sig) {
  double pm = 1.0, p = d[0] - sig;
  bool negp = dneg(p) || dzero(p);
  int cnt = negp ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    const double pn = fma(d[i] - sig, p, -e2[i - 1] * pm);
    pm = p;
    p = pn;
    const bool neg = dzero(p) ? !negp : dneg(p);
    cnt += neg != negp;
    negp = neg;
    if ((i & 7) == 0) {
      const int ex = max(dexp(p), dexp(pm));
      if (ex > 1023 + 600) {
        p *= 0x1p-600;
        pm *= 0x1p-600;
      } else if (ex < 1023 - 600 && ex > 0) {
        p *= 0x1p600;
        pm *= 0x1p600;
      }
    }
  }
  return cnt;
}

// The same count in single precision, in ratio form q_i = p_i / p_{i-1}
// (a ratio below tiny in magnitude is taken as -tiny).  It is exact for a
// matrix within a few single-precision units of ||T|| of T.
__device__ __forceinline__ int sturm_count_f(const float* d, const float* e2, int n, float sig,
                                             float tiny) {
  float q = d[0] - sig;
  if (fabsf(q) < tiny) q = -tiny;
  int cnt = q < 0.f ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - sig) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < tiny) q = -tiny;
    cnt += q < 0.f ? 1 : 0;
  }
  return cnt;
}

// One multisection round for the t-th smallest eigenvalue (t = 0, 1, ...):
// lanes count at 32 interior points of [lo, hi]; the bracket shrinks 33x.
// Brackets of eigenvalues 1 and n - 1 are narrowed from the same counts.
struct Bracket {
  double lo, hi;
};
__device__ __forceinline__ void shrink(Bracket& b, unsigned above, double sig) {
  const int first = above ? __ffs(above) - 1 : 32;
  const double slo = __shfl_sync(0xffffffffu, sig, first > 0 ? first - 1 : 0);
  const double shi = __shfl_sync(0xffffffffu, sig, first < 32 ? first : 31);
  if (first > 0) b.lo = fmax(b.lo, slo);
  if (first < 32) b.hi = fmin(b.hi, shi);
}
// One round on bracket t; the counts narrow all nb brackets (target
// eigenvalue index which[m] each).  SINGLE: counts in single precision at
// shifts rounded to single precision.
template <bool SINGLE>
__device__ void multisect(const TriWs& W, int n, int t, Bracket* br, int nb, const int* which,
                          float tiny_f) {
  const int lane = threadIdx.x & 31;
  const double h = (br[t].hi - br[t].lo) * (1.0 / 33.0);
  double sig = fma(h, (double)(lane + 1), br[t].lo);
  int c;
  if (SINGLE) {
    const float sf = (float)sig;
    sig = (double)sf;
    c = sturm_count_f(W.df, W.e2f, n, sf, tiny_f);
  } else {
    c = sturm_count(W.d, W.e2, n, sig);
  }
  for (int m = 0; m < nb; ++m) {
    const unsigned above = __ballot_sync(0xffffffffu, c > which[m]);
    shrink(br[m], above, sig);
  }
}

// 3. LU of the tridiagonal T - sig I with row interchanges (lane 0 only);
// pivots below tiny = u ||T|| in magnitude become +-tiny.  u0 keeps the
// reciprocals of U's diagonal.
__device__ __forceinline__ double rcp_safe(double x) {
  return fabs(x) > 1e-30 && fabs(x) < 1e30 ? rcp_d(x) : 1.0 / x;
}
__device__ __forceinline__ double rsqrt_safe(double x) {
  return x > 1e-30 && x < 1e30 ? rsqrt_d(x) : 1.0 / sqrt(x);
}
__device__ __forceinline__ double clamp_pivot(double x, double tiny) {
  return fabs(x) >= tiny ? x : (dneg(x) ? -tiny : tiny);
}
__device__ __forceinline__ float rcp_safe(float x) { return 1.0f / x; }
__device__ __forceinline__ float clamp_pivot(float x, float tiny) {
  return fabsf(x) >= tiny ? x : (x < 0.f ? -tiny : tiny);
}
template <typename R>
__device__ void tri_lu(const R* d, const R* e, R* u0, R* u1, R* u2, R* lm, int* pv, int n, R sig,
                       R tiny) {
  if ((threadIdx.x & 31) != 0) return;
  for (int i = 0; i < n; ++i) {
    u0[i] = d[i] - sig;
    u1[i] = i + 1 < n ? e[i] : R(0);
    u2[i] = R(0);
  }
  for (int i = 0; i + 1 < n; ++i) {
    const R sub = e[i];   // element (i + 1, i)
    const R piv = u0[i];
    if (fabs(piv) >= fabs(sub)) {
      const R r = rcp_safe(clamp_pivot(piv, tiny));
      const R m = sub * r;
      lm[i] = m;
      pv[i] = 0;
      u0[i] = r;
      u0[i + 1] -= m * u1[i];
    } else {
      const R r = rcp_safe(sub);
      const R m = piv * r;
      const R a1 = u0[i + 1], b1 = u1[i + 1];
      lm[i] = m;
      pv[i] = 1;
      u0[i] = r;
      u0[i + 1] = u1[i] - m * a1;
      u1[i + 1] = -m * b1;
      u1[i] = a1;
      u2[i] = b1;
    }
  }
  u0[n - 1] = rcp_safe(clamp_pivot(u0[n - 1], tiny));
}
__device__ __forceinline__ void tri_lu(const TriWs& W, int n, double sig, double tiny) {
  tri_lu<double>(W.d, W.e, W.u0, W.u1, W.u2, W.lm, W.piv, n, sig, tiny);
}

// Solve (T - sig I) z = b in place from tri_lu's factors (lane 0 only).
template <typename R, typename V>
__device__ void tri_solve(const R* u0, const R* u1, const R* u2, const R* lm, const int* pv, int n,
                          V* b) {
  if ((threadIdx.x & 31) != 0) return;
  for (int i = 0; i + 1 < n; ++i) {
    if (pv[i]) {
      const V t = b[i];
      b[i] = b[i + 1];
      b[i + 1] = t;
    }
    b[i + 1] = b[i + 1] - lm[i] * b[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    V v = b[i];
    if (i + 1 < n) v = v - u1[i] * b[i + 1];
    if (i + 2 < n) v = v - u2[i] * b[i + 2];
    b[i] = u0[i] * v;
  }
}
__device__ __forceinline__ void tri_solve(const TriWs& W, int n, cd* b) {
  tri_solve<double, cd>(W.u0, W.u1, W.u2, W.lm, W.piv, n, b);
}

// Apply Q (back = true: b <- Q b) or Q^H (b <- Q^H b) to b (n, complex V).
template <typename E, typename V>
__device__ void tri_apply_q(const E* A, const E* tau, int n, V* b, bool back) {
  using R = typename RealOf<V>::type;
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int s = 0; s + 1 < n; ++s) {
    const int k = back ? n - 2 - s : s;
    const V tk = to_v(tau[k], V());
    if (tk.re == R(0) && tk.im == R(0)) continue;
    const E* vk = A + (size_t)k * n;
    V acc = mk(R(0), R(0));
    for (int i = lane; i < n; i += 32)
      if (i > k) cfmac(acc, to_v(vk[i], V()), b[i]);   // v^H b
    acc = mk(warp_sum(acc.re), warp_sum(acc.im));
    const V f = (back ? tk : conj(tk)) * acc;
    __syncwarp();
    for (int i = lane; i < n; i += 32)
      if (i > k) b[i] = b[i] - f * to_v(vk[i], V());
    __syncwarp();
  }
}

// Real reflectors on a real vector (real samples): half the work of the
// complex form.
__device__ void tri_apply_q_r(const double* A, const double* tau, int n, double* b, bool back) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int s = 0; s + 1 < n; ++s) {
    const int k = back ? n - 2 - s : s;
    const double tk = tau[k];
    if (tk == 0.0) continue;
    const double* vk = A + (size_t)k * n;
    double acc = 0.0;
    for (int i = lane; i < n; i += 32)
      if (i > k) acc = fma(vk[i], b[i], acc);
    const double f = tk * warp_sum(acc);
    __syncwarp();
    for (int i = lane; i < n; i += 32)
      if (i > k) b[i] = fma(-f, vk[i], b[i]);
    __syncwarp();
  }
}
__device__ __forceinline__ double tri_norm2_r(const double* b, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s = fma(b[i], b[i], s);
  return warp_sum(s);
}

__device__ __forceinline__ double tri_norm2(const cd* b, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < n; i += 32) s += abs2(b[i]);
  return warp_sum(s);
}

struct TriResult {
  double lam_min, lam_2, lam_max;   // eigenvalues of G (T's, scaled back)
  double theta;                     // x^H G x
  int near_degenerate;              // lam_2 - lam_min <= 1e-4 lam_max
};

// CTA- or warp-wide barrier.
template <bool BLOCK> __device__ __forceinline__ void team_sync() {
  if (BLOCK) __syncthreads();
  else __syncwarp();
}

// Steps 1-4 by one warp: T, the eigenvalue brackets, x.  Returns the number
// of refinement steps to take; fills res (eigenvalues), gs (the power-of-two
// scale of G) and tnorm.
template <typename E>
__device__ int tri_solve_lead(const TriWs& W, const cd* G, int n, int steps_far, int steps_near,
                              double refine_gap, TriResult& res, double& gs, double& tnorm,
                              long long* tk, bool prereduced = false) {
  const int lane = threadIdx.x & 31;
  E* A = (E*)W.A;
  E* tau = (E*)W.tau;
  // scale by a power of two so that the largest diagonal entry is in [1/2, 1)
  double gmax = 0.0;
  for (int i = lane; i < n; i += 32) gmax = fmax(gmax, G[(size_t)i * n + i].re);
  gmax = warp_max(gmax);
  if (!(gmax > 0.0)) {   // zero matrix: every vector is a null vector
    for (int i = lane; i < n; i += 32) W.x[i] = mk(i == 0 ? 1.0 : 0.0, 0.0);
    __syncwarp();
    res.lam_min = res.lam_2 = res.lam_max = 0.0;
    res.near_degenerate = 1;
    gs = 1.0;
    tnorm = 0.0;
    return 0;
  }
  int ex;
  frexp(gmax, &ex);
  gs = ldexp(1.0, ex);
  const double igs = ldexp(1.0, -ex);
  if (!prereduced) {   // else the caller's CTA has reduced G * igs already
    for (int idx = lane; idx < n * n; idx += 32) {
      if constexpr (sizeof(E) == sizeof(double)) A[idx] = mk_e<E, double>(G[idx].re * igs, 0.0);
      else A[idx] = mk_e<E, double>(G[idx].re * igs, G[idx].im * igs);
    }
    __syncwarp();
    if (tk && lane == 0) tk[0] = clock64();
    tri_reduce<E>(A, tau, (E*)W.w, W.d, W.e, n);
    if (tk && lane == 0) tk[1] = clock64();
  }
  // Gershgorin interval of T; single-precision copies
  double glo = 1e300, ghi = -1e300;
  for (int i = lane; i < n; i += 32) {
    const double rad = (i > 0 ? fabs(W.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(W.e[i]) : 0.0);
    glo = fmin(glo, W.d[i] - rad);
    ghi = fmax(ghi, W.d[i] + rad);
    const double e2 = i + 1 < n ? W.e[i] * W.e[i] : 0.0;
    W.e2[i] = e2;
    W.df[i] = (float)W.d[i];
    W.e2f[i] = (float)e2;
  }
  glo = -warp_max(-glo);
  ghi = warp_max(ghi);
  tnorm = fmax(fabs(glo), fabs(ghi));
  const double eps = 2.220446049250313e-16;
  glo -= 4.0 * eps * tnorm + 1e-300;
  ghi += 4.0 * eps * tnorm + 1e-300;
  __syncwarp();
  // 2. brackets of eigenvalues 0, 1 and n - 1
  const int which[3] = {0, n > 1 ? 1 : 0, n - 1};
  Bracket br[3] = {{glo, ghi}, {glo, ghi}, {glo, ghi}};
  // single-precision rounds while a bracket is wider than its floor
  const double fl = 1e-5 * tnorm;
  const float tiny_f = (float)(1e-30 * fmax(tnorm, 1e-8));
  for (int round = 0; round < 12; ++round) {
    int t = -1;
    for (int m = 2; m >= 0; --m)
      if (br[m].hi - br[m].lo > fl) t = m;
    if (t < 0) break;
    multisect<true>(W, n, t, br, 3, which, tiny_f);
  }
  // widen by the single-precision error bound; check the ends in double
  // precision (a wrong end falls back to the Gershgorin interval)
  for (int m = 0; m < 3; ++m) {
    br[m].lo = fmax(glo, br[m].lo - 4e-6 * tnorm);
    br[m].hi = fmin(ghi, br[m].hi + 4e-6 * tnorm);
  }
  {
    const int m = lane % 3, end = (lane / 3) & 1;
    const double sig = end ? br[m].hi : br[m].lo;
    const int c = lane < 6 ? sturm_count(W.d, W.e2, n, sig) : 0;
    const bool bad = lane < 6 && (end ? c <= which[m] : c > which[m]);
    const unsigned badm = __ballot_sync(0xffffffffu, bad);
    for (int m2 = 0; m2 < 3; ++m2)
      if (badm & (0x9u << m2)) br[m2] = Bracket{glo, ghi};
  }
  const double tol_abs = 8.0 * eps * tnorm;
  for (int round = 0; round < 40; ++round) {
    // isolated well enough: the inverse iteration contracts by 1e-4 per step
    const double w0 = br[0].hi - br[0].lo;
    if (w0 <= tol_abs || (n > 1 && br[1].lo > br[0].hi && w0 <= 1e-4 * (br[1].lo - br[0].hi)))
      break;
    multisect<false>(W, n, 0, br, 3, which, tiny_f);
  }
  if (n > 1) {
    for (int round = 0; round < 40; ++round) {
      const double w1 = br[1].hi - br[1].lo;
      if (w1 <= fmax(tol_abs, 1e-5 * fabs(br[1].hi))) break;
      multisect<false>(W, n, 1, br, 3, which, tiny_f);
    }
  }
  for (int round = 0; round < 40; ++round) {
    const double w2 = br[2].hi - br[2].lo;
    if (w2 <= fmax(tol_abs, 1e-7 * fabs(br[2].hi))) break;
    multisect<false>(W, n, 2, br, 3, which, tiny_f);
  }
  if (tk && lane == 0) tk[2] = clock64();
  const double lam0 = 0.5 * (br[0].lo + br[0].hi);
  const double lam1 = n > 1 ? 0.5 * (br[1].lo + br[1].hi) : lam0;
  const double lamn = 0.5 * (br[2].lo + br[2].hi);
  // 3. inverse iteration (three steps) from a fixed start vector; 4. x = Q y
  tri_lu(W, n, lam0, eps * tnorm);
  if constexpr (sizeof(E) == sizeof(double)) {   // real: real vectors throughout
    double* y = (double*)W.z;
    for (int i = lane; i < n; i += 32) y[i] = 1.0 + 0.25 * (double)((i * 7) % 5);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      tri_solve<double, double>(W.u0, W.u1, W.u2, W.lm, W.piv, n, y);
      __syncwarp();
      const double nz = tri_norm2_r(y, n);
      const double sc = nz > 0.0 ? rsqrt_safe(nz) : 1.0;
      for (int i = lane; i < n; i += 32) y[i] = sc * y[i];
      __syncwarp();
    }
    tri_apply_q_r((const double*)A, (const double*)tau, n, y, true);
    const double sc = rsqrt_safe(tri_norm2_r(y, n));
    for (int i = lane; i < n; i += 32) W.x[i] = mk(sc * y[i], 0.0);
    __syncwarp();
  } else {
    for (int i = lane; i < n; i += 32) W.z[i] = mk(1.0 + 0.25 * (double)((i * 7) % 5), 0.0);
    __syncwarp();
    for (int it = 0; it < 3; ++it) {
      tri_solve(W, n, W.z);
      __syncwarp();
      const double nz = tri_norm2(W.z, n);
      const double sc = nz > 0.0 ? rsqrt_safe(nz) : 1.0;
      for (int i = lane; i < n; i += 32) W.z[i] = sc * W.z[i];
      __syncwarp();
    }
    for (int i = lane; i < n; i += 32) W.x[i] = W.z[i];
    tri_apply_q<E, cd>(A, tau, n, W.x, true);
    const double sc = rsqrt_safe(tri_norm2(W.x, n));
    for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
    __syncwarp();
  }
  if (tk && lane == 0) tk[3] = clock64();
  res.lam_min = gs * lam0;
  res.lam_2 = gs * lam1;
  res.lam_max = gs * lamn;
  res.near_degenerate = n > 1 && (lam1 - lam0) <= 1e-4 * lamn ? 1 : 0;
  const bool near = n > 1 && (lam1 - lam0) <= refine_gap * lamn;
  return near ? steps_near : steps_far;
}

// Steps 1-4 in single precision, then Newton steps in Olsen's form against
// G itself: the residual G x - theta x in double precision, the correction
// equation solved through the single-precision T (contraction ~n u ||T|| /
// gap per step), until the correction stops shrinking or falls below 1e-10.
// For complex matrices whose two smallest eigenvalues single precision
// separates by more than 3e-5 lambda_max (contraction <~ 0.1 per step, at
// most 12 steps), or separates at all with a gap above 1e-5 lambda_max (at
// most 24 steps, which must bring the correction below 1e-9); returns false,
// having changed nothing but the work area, for the others (they take
// tri_solve_lead).
// Gx: a float-float copy of G (or null): the Newton steps' residual G x is
// then formed on the single-precision units (~1e-14) instead of in double.
__device__ bool tri_solve_lead_sp(const TriWs& W, const cd* G, int n, TriResult& res, double& gs,
                                  double& tnorm, long long* tk, bool prereduced = false,
                                  const cfx* Gx = nullptr) {
  const int lane = threadIdx.x & 31;
  cf* A = (cf*)W.A;
  cf* tau = (cf*)W.tau;
  float* d = W.df;
  float* e = (float*)W.e;
  float* u0 = (float*)W.u0;
  float* u1 = (float*)W.u1;
  float* u2 = (float*)W.u2;
  float* lm = (float*)W.lm;
  double gmax = 0.0;
  for (int i = lane; i < n; i += 32) gmax = fmax(gmax, G[(size_t)i * n + i].re);
  gmax = warp_max(gmax);
  if (!(gmax > 0.0)) return false;
  int ex;
  frexp(gmax, &ex);
  gs = ldexp(1.0, ex);
  const double igs = ldexp(1.0, -ex);
  if (!prereduced) {   // else the CTA has reduced the same single-precision copy
    const float igsf = (float)igs;
    for (int idx = lane; idx < n * n; idx += 32)
      A[idx] = mk((float)G[idx].re * igsf, (float)G[idx].im * igsf);
    __syncwarp();
    if (tk && lane == 0) tk[0] = clock64();
    tri_reduce<cf>(A, tau, (cf*)W.w, d, e, n);
    if (tk && lane == 0) tk[1] = clock64();
  }
  float glo = 1e30f, ghi = -1e30f;
  for (int i = lane; i < n; i += 32) {
    const float rad = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i + 1 < n ? fabsf(e[i]) : 0.f);
    glo = fminf(glo, d[i] - rad);
    ghi = fmaxf(ghi, d[i] + rad);
    W.e2f[i] = i + 1 < n ? e[i] * e[i] : 0.f;
  }
  glo = -warp_max(-glo);
  ghi = warp_max(ghi);
  tnorm = fmax(fabs((double)glo), fabs((double)ghi));
  __syncwarp();
  const int which[3] = {0, 1, n - 1};
  const double eb = 4e-6 * tnorm;     // single-precision error bound of the counts
  Bracket br[3];
  for (int m = 0; m < 3; ++m) br[m] = Bracket{(double)glo - eb, (double)ghi + eb};
  const float tiny_f = (float)(1e-30 * fmax(tnorm, 1e-8));
  for (int round = 0; round < 14; ++round) {
    int t = -1;
    for (int m = 2; m >= 0; --m)
      if (br[m].hi - br[m].lo > 0.25 * eb) t = m;
    if (t < 0) break;
    multisect<true>(W, n, t, br, 3, which, tiny_f);
  }
  const double lam0 = 0.5 * (br[0].lo + br[0].hi), lam1 = 0.5 * (br[1].lo + br[1].hi);
  const double lamn = 0.5 * (br[2].lo + br[2].hi);
  // separated beyond the error bounds?  Well beyond (3e-5 lambda_max): at
  // most 12 Newton steps, contraction <~ 0.1.  Narrowly (apart within the
  // bounds, gap above 1e-5 lambda_max, contraction <~ 0.3): up to 24 steps,
  // and the double-precision solve after all unless they converge.
  const double sep = (br[1].lo - eb) - (br[0].hi + eb);
  const bool wide = sep > 3e-5 * lamn;
  if (!wide && !(sep > 0.0 && lam1 - lam0 > 1e-5 * lamn)) {
#ifdef CBP_PHASE_TIMING
    if (lane == 0)
      printf("sp-reject n=%d lam0/lamn %.3e lam1/lamn %.3e eb/lamn %.3e\n", n, lam0 / lamn, lam1 / lamn,
             eb / lamn);
#endif
    return false;
  }
  if (tk && lane == 0) tk[2] = clock64();
  // inverse iteration in single precision (three steps)
  tri_lu<float>(d, e, u0, u1, u2, lm, W.piv, n, (float)lam0, (float)(1.2e-7 * tnorm));
  cf* y = (cf*)W.z;
  for (int i = lane; i < n; i += 32) y[i] = mk(1.0f + 0.25f * (float)((i * 7) % 5), 0.f);
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    tri_solve<float, cf>(u0, u1, u2, lm, W.piv, n, y);
    __syncwarp();
    float s2 = 0.f;
    for (int i = lane; i < n; i += 32) s2 += abs2(y[i]);
    s2 = warp_sum(s2);
    const float sc = s2 > 0.f ? rsqrtf(s2) : 1.f;
    for (int i = lane; i < n; i += 32) y[i] = sc * y[i];
    __syncwarp();
  }
  // Q explicitly (lane i builds column i: H_0 ... H_{n-2} e_i), row stride n + 1
  cf* Q = A + (size_t)n * n;
  const int lq = n + 1;
  for (int i = lane; i < n; i += 32) {
    for (int j = 0; j < n; ++j) Q[(size_t)j * lq + i] = mk(j == i ? 1.f : 0.f, 0.f);
    for (int k = n - 2; k >= 0; --k) {
      const cf tk = tau[k];
      if (tk.re == 0.f && tk.im == 0.f) continue;
      const cf* vk = A + (size_t)k * n;
      cf s0 = mk(0.f, 0.f), s1 = mk(0.f, 0.f);
      int j = k + 1;
      for (; j + 1 < n; j += 2) {
        cfmac(s0, vk[j], Q[(size_t)j * lq + i]);
        cfmac(s1, vk[j + 1], Q[(size_t)(j + 1) * lq + i]);
      }
      if (j < n) cfmac(s0, vk[j], Q[(size_t)j * lq + i]);
      const cf f = tk * (s0 + s1);
      for (int jj = k + 1; jj < n; ++jj) Q[(size_t)jj * lq + i] = Q[(size_t)jj * lq + i] - f * vk[jj];
    }
  }
  __syncwarp();
  // x = Q y
  for (int i = lane; i < n; i += 32) {
    cf acc = mk(0.f, 0.f);
    for (int j = 0; j < n; ++j) cfma(acc, Q[(size_t)i * lq + j], y[j]);
    W.x[i] = mk((double)acc.re, (double)acc.im);
  }
  __syncwarp();
  {
    const double sc = rsqrt_safe(tri_norm2(W.x, n));
    for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
    __syncwarp();
  }
  if (tk && lane == 0) tk[3] = clock64();
  // Newton steps against G
  cf* rt = (cf*)W.q;          // Q^H r, then u
  cf* zt = rt + n;            // Q^H x, then z
  cf* yt = (cf*)W.z;          // Q^H x
  cf* yq = yt + n;            // x in single precision
  cf* rq = (cf*)W.r;          // r in single precision, then d~
  double dprev = 1e300, dn = 1e300;
  const int max_it = wide ? 12 : 24;
  const double stall = wide ? 0.25 : 0.5;
  for (int it = 0; it < max_it; ++it) {
    cd gx[2];
    cd th = mk(0.0, 0.0);
    if (Gx) {
      cfx* xx = (cfx*)W.part;   // x in float-float (the reduction's scratch is free)
      for (int i = lane; i < n; i += 32) xx[i] = cfx_of(W.x[i]);
      __syncwarp();
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int i = lane + 32 * c;
        gx[c] = mk(0.0, 0.0);
        if (i < n) {
          cfx_acc acc;
          for (int j = 0; j < n; ++j) acc.macc(Gx[(size_t)j * n + i], xx[j]);   // (G x)_i
          gx[c] = cfx_val(acc.value());
          cfmac(th, W.x[i], gx[c]);
        }
      }
      __syncwarp();
    } else {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int i = lane + 32 * c;
        gx[c] = mk(0.0, 0.0);
        if (i < n) {
          for (int j = 0; j < n; ++j) cfmac(gx[c], G[(size_t)j * n + i], W.x[j]);   // (G x)_i
          cfmac(th, W.x[i], gx[c]);
        }
      }
    }
    const double theta = warp_sum(th.re);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = lane + 32 * c;
      if (i < n) {
        const cd r = gx[c] - theta * W.x[i];
        rq[i] = mk((float)r.re, (float)r.im);
        yq[i] = mk((float)W.x[i].re, (float)W.x[i].im);
      }
    }
    __syncwarp();
    // r~ = Q^H r, y~ = Q^H x (lane i: column i of Q)
    for (int i = lane; i < n; i += 32) {
      cf a0 = mk(0.f, 0.f), a1 = mk(0.f, 0.f);
      for (int j = 0; j < n; ++j) {
        const cf q = Q[(size_t)j * lq + i];
        cfmac(a0, q, yq[j]);
        cfmac(a1, q, rq[j]);
      }
      yt[i] = a0;
      zt[i] = a0;
      rt[i] = a1;
    }
    tri_lu<float>(d, e, u0, u1, u2, lm, W.piv, n, (float)(theta * igs), (float)(1.2e-7 * tnorm));
    __syncwarp();
    tri_solve<float, cf>(u0, u1, u2, lm, W.piv, n, rt);   // u
    tri_solve<float, cf>(u0, u1, u2, lm, W.piv, n, zt);   // z
    __syncwarp();
    cf nu = mk(0.f, 0.f), de = mk(0.f, 0.f);
    for (int i = lane; i < n; i += 32) {
      cfmac(nu, yt[i], rt[i]);
      cfmac(de, yt[i], zt[i]);
    }
    nu = mk(warp_sum(nu.re), warp_sum(nu.im));
    de = mk(warp_sum(de.re), warp_sum(de.im));
    const float dd = abs2(de);
    const cf epsn = dd > 0.f ? (1.0f / dd) * (nu * conj(de)) : mk(0.f, 0.f);
    const float ig = (float)igs;
    for (int i = lane; i < n; i += 32) rq[i] = ig * (epsn * zt[i] - rt[i]);
    __syncwarp();
    float d2 = 0.f;
    for (int i = lane; i < n; i += 32) {   // d = Q d~ (lane i: row i of Q)
      cf acc = mk(0.f, 0.f);
      for (int j = 0; j < n; ++j) cfma(acc, Q[(size_t)i * lq + j], rq[j]);
      W.x[i] = W.x[i] + mk((double)acc.re, (double)acc.im);
      d2 += abs2(acc);
    }
    d2 = warp_sum(d2);
    __syncwarp();
    const double sc = rsqrt_safe(tri_norm2(W.x, n));
    for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
    __syncwarp();
    dn = sqrt((double)d2);
    if (dn < 1e-10 || dn > stall * dprev) break;
    dprev = dn;
  }
  if (!wide && !(dn < 1e-9)) {
#ifdef CBP_PHASE_TIMING
    if (lane == 0) printf("sp-narrow-fail n=%d last correction %.3e\n", n, dn);
#endif
    return false;
  }
  res.lam_min = gs * lam0;
  res.lam_2 = gs * lam1;
  res.lam_max = gs * lamn;
  res.near_degenerate = (lam1 - lam0) <= 1e-4 * lamn ? 1 : 0;
  return true;
}

// One refinement step by the lead warp after r = (exact operator) x: Olsen's
// correction through T (step 5).
template <typename E>
__device__ void tri_olsen(const TriWs& W, int n, double gs, double tnorm) {
  const int lane = threadIdx.x & 31;
  const E* A = (const E*)W.A;
  const E* tau = (const E*)W.tau;
  const double eps = 2.220446049250313e-16, igs = 1.0 / gs;
  if constexpr (sizeof(E) == sizeof(double)) {   // real sample: real vectors
    double th = 0.0;
    for (int i = lane; i < n; i += 32) th = fma(W.x[i].re, W.r[i].re, th);
    const double theta = warp_sum(th);
    double* ru = (double*)W.q;        // Q^T r, then u
    double* yt = ru + n;              // Q^T x
    double* zt = (double*)W.z;        // z, then the correction
    for (int i = lane; i < n; i += 32) {
      ru[i] = W.r[i].re - theta * W.x[i].re;
      yt[i] = W.x[i].re;
    }
    tri_apply_q_r((const double*)A, (const double*)tau, n, ru, false);
    tri_apply_q_r((const double*)A, (const double*)tau, n, yt, false);
    tri_lu(W, n, theta * igs, eps * tnorm);
    for (int i = lane; i < n; i += 32) zt[i] = yt[i];
    __syncwarp();
    tri_solve<double, double>(W.u0, W.u1, W.u2, W.lm, W.piv, n, ru);
    tri_solve<double, double>(W.u0, W.u1, W.u2, W.lm, W.piv, n, zt);
    __syncwarp();
    double nu = 0.0, de = 0.0;
    for (int i = lane; i < n; i += 32) {
      nu = fma(yt[i], ru[i], nu);
      de = fma(yt[i], zt[i], de);
    }
    nu = warp_sum(nu);
    de = warp_sum(de);
    const double ep = de != 0.0 ? nu / de : 0.0;
    for (int i = lane; i < n; i += 32) zt[i] = igs * (ep * zt[i] - ru[i]);
    tri_apply_q_r((const double*)A, (const double*)tau, n, zt, true);
    for (int i = lane; i < n; i += 32) W.x[i] = mk(W.x[i].re + zt[i], 0.0);
    __syncwarp();
    const double sc = rsqrt_safe(tri_norm2(W.x, n));
    for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
    __syncwarp();
    return;
  }
  cd th = mk(0.0, 0.0);
  for (int i = lane; i < n; i += 32) cfmac(th, W.x[i], W.r[i]);
  const double theta = warp_sum(th.re);
  for (int i = lane; i < n; i += 32) {
    W.r[i] = W.r[i] - theta * W.x[i];
    W.q[i] = W.x[i];
  }
  // to T coordinates: r~ = Q^H r, y~ = Q^H x
  tri_apply_q<E, cd>(A, tau, n, W.r, false);
  tri_apply_q<E, cd>(A, tau, n, W.q, false);
  tri_lu(W, n, theta * igs, eps * tnorm);
  for (int i = lane; i < n; i += 32) W.z[i] = W.q[i];
  __syncwarp();
  tri_solve(W, n, W.r);    // u = (T - theta)^{-1} r~
  tri_solve(W, n, W.z);    // z = (T - theta)^{-1} y~
  __syncwarp();
  cd nu = mk(0.0, 0.0), de = mk(0.0, 0.0);
  for (int i = lane; i < n; i += 32) {
    cfmac(nu, W.q[i], W.r[i]);
    cfmac(de, W.q[i], W.z[i]);
  }
  nu = mk(warp_sum(nu.re), warp_sum(nu.im));
  de = mk(warp_sum(de.re), warp_sum(de.im));
  const double dd = abs2(de);
  const cd epsn = dd > 0.0 ? (1.0 / dd) * (nu * conj(de)) : mk(0.0, 0.0);
  // d = (-u + eps z) / gs in T coordinates, then back
  for (int i = lane; i < n; i += 32) W.z[i] = igs * (epsn * W.z[i] - W.r[i]);
  tri_apply_q<E, cd>(A, tau, n, W.z, true);
  for (int i = lane; i < n; i += 32) W.x[i] = W.x[i] + W.z[i];
  __syncwarp();
  const double sc = rsqrt_safe(tri_norm2(W.x, n));
  for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
  __syncwarp();
}

// The same step for a real sample by a CTA of three or more warps: the two
// projections onto T's basis and the factorisation of T - theta run on three
// warps at once, the two solves on two, the rest on the lead warp (the same
// arithmetic as tri_olsen<double>, in the same order within each chain).
__device__ void tri_olsen_real_block(const TriWs& W, int n, double gs, double tnorm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* A = (const double*)W.A;
  const double* tau = (const double*)W.tau;
  const double eps = 2.220446049250313e-16, igs = 1.0 / gs;
  double* ru = (double*)W.q;        // Q^T r, then u
  double* yt = ru + n;              // Q^T x
  double* zt = (double*)W.z;        // z, then the correction
  double th = 0.0;
  for (int i = lane; i < n; i += 32) th = fma(W.x[i].re, W.r[i].re, th);
  const double theta = warp_sum(th);
  if (warp == 0) {
    for (int i = lane; i < n; i += 32) ru[i] = W.r[i].re - theta * W.x[i].re;
    tri_apply_q_r(A, tau, n, ru, false);
  } else if (warp == 1) {
    for (int i = lane; i < n; i += 32) yt[i] = W.x[i].re;
    tri_apply_q_r(A, tau, n, yt, false);
    for (int i = lane; i < n; i += 32) zt[i] = yt[i];
    __syncwarp();
  } else if (warp == 2) {
    tri_lu(W, n, theta * igs, eps * tnorm);
  }
  __syncthreads();
  if (warp == 0) tri_solve<double, double>(W.u0, W.u1, W.u2, W.lm, W.piv, n, ru);
  else if (warp == 1) tri_solve<double, double>(W.u0, W.u1, W.u2, W.lm, W.piv, n, zt);
  __syncthreads();
  if (warp == 0) {
    double nu = 0.0, de = 0.0;
    for (int i = lane; i < n; i += 32) {
      nu = fma(yt[i], ru[i], nu);
      de = fma(yt[i], zt[i], de);
    }
    nu = warp_sum(nu);
    de = warp_sum(de);
    const double ep = de != 0.0 ? nu / de : 0.0;
    for (int i = lane; i < n; i += 32) zt[i] = igs * (ep * zt[i] - ru[i]);
    tri_apply_q_r(A, tau, n, zt, true);
    for (int i = lane; i < n; i += 32) W.x[i] = mk(W.x[i].re + zt[i], 0.0);
    __syncwarp();
    const double sc = rsqrt_safe(tri_norm2(W.x, n));
    for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
    __syncwarp();
  }
  __syncthreads();
}

// ------------------------------------------------------------------------
// Float-float forms of the real samples' steps 2-5 (mixed path): on this GPU
// a double-precision instruction holds a scheduler's double unit for ~64
// cycles, and these steps are chains of them on one lane or one warp.  The
// same algorithms with float-float values (~48 bits) on the single-precision
// units; T's eigenvalues come out to ~1e-13 ||T||, the vector from inverse
// iteration and the Olsen step as before.

// Sturm count of T - sig I from the leading minors p_i (product form),
// rescaled by powers of two when they leave [2^-60, 2^60].
__device__ __forceinline__ int sturm_count_x(const fx* d, const fx* e2, int n, fx sig) {
  fx pm = {1.f, 0.f}, p = fx_sub(d[0], sig);
  bool negp = fx_neg_sign(p) || fx_is_zero(p);
  int cnt = negp ? 1 : 0;
  for (int i = 1; i < n; ++i) {
    const fx pn = fx_sub(fx_mul(fx_sub(d[i], sig), p), fx_mul(e2[i - 1], pm));
    pm = p;
    p = pn;
    const bool neg = fx_is_zero(p) ? !negp : fx_neg_sign(p);
    cnt += neg != negp;
    negp = neg;
    const float a = fmaxf(fabsf(p.hi), fabsf(pm.hi));
    if (a > 0x1p60f) {
      p = fx_ldexp(p, -60);
      pm = fx_ldexp(pm, -60);
    } else if (a < 0x1p-60f && a > 0.f) {
      p = fx_ldexp(p, 60);
      pm = fx_ldexp(pm, 60);
    }
  }
  return cnt;
}

__device__ void multisect_x(const fx* d, const fx* e2, int n, int t, Bracket* br, int nb,
                            const int* which) {
  const int lane = threadIdx.x & 31;
  const double h = (br[t].hi - br[t].lo) * (1.0 / 33.0);
  const double sig = fma(h, (double)(lane + 1), br[t].lo);
  const int c = sturm_count_x(d, e2, n, fx_of(sig));
  for (int m = 0; m < nb; ++m) {
    const unsigned above = __ballot_sync(0xffffffffu, c > which[m]);
    shrink(br[m], above, sig);
  }
}

__device__ __forceinline__ fx fx_clamp_pivot(fx x, float tiny) {
  return fabsf(x.hi) >= tiny ? x : fx{fx_neg_sign(x) ? -tiny : tiny, 0.f};
}
// LU of T - sig I with row interchanges (lane 0), as tri_lu
__device__ void tri_lu_x(const fx* d, const fx* e, fx* u0, fx* u1, fx* u2, fx* lm, int* pv, int n,
                         fx sig, float tiny) {
  if ((threadIdx.x & 31) != 0) return;
  const fx one = {1.f, 0.f}, zero = {0.f, 0.f};
  for (int i = 0; i < n; ++i) {
    u0[i] = fx_sub(d[i], sig);
    u1[i] = i + 1 < n ? e[i] : zero;
    u2[i] = zero;
  }
  for (int i = 0; i + 1 < n; ++i) {
    const fx sub = e[i];
    const fx piv = u0[i];
    if (fabsf(piv.hi) >= fabsf(sub.hi)) {
      const fx r = fx_div(one, fx_clamp_pivot(piv, tiny));
      const fx m = fx_mul(sub, r);
      lm[i] = m;
      pv[i] = 0;
      u0[i] = r;
      u0[i + 1] = fx_sub(u0[i + 1], fx_mul(m, u1[i]));
    } else {
      const fx r = fx_div(one, sub);
      const fx m = fx_mul(piv, r);
      const fx a1 = u0[i + 1], b1 = u1[i + 1];
      lm[i] = m;
      pv[i] = 1;
      u0[i] = r;
      u0[i + 1] = fx_sub(u1[i], fx_mul(m, a1));
      u1[i + 1] = fx_neg(fx_mul(m, b1));
      u1[i] = a1;
      u2[i] = b1;
    }
  }
  u0[n - 1] = fx_div(one, fx_clamp_pivot(u0[n - 1], tiny));
}
__device__ void tri_solve_x(const fx* u0, const fx* u1, const fx* u2, const fx* lm, const int* pv,
                            int n, fx* b) {
  if ((threadIdx.x & 31) != 0) return;
  for (int i = 0; i + 1 < n; ++i) {
    if (pv[i]) {
      const fx t = b[i];
      b[i] = b[i + 1];
      b[i + 1] = t;
    }
    b[i + 1] = fx_sub(b[i + 1], fx_mul(lm[i], b[i]));
  }
  for (int i = n - 1; i >= 0; --i) {
    fx v = b[i];
    if (i + 1 < n) v = fx_sub(v, fx_mul(u1[i], b[i + 1]));
    if (i + 2 < n) v = fx_sub(v, fx_mul(u2[i], b[i + 2]));
    b[i] = fx_mul(u0[i], v);
  }
}
__device__ __forceinline__ fx warp_sum_x(fx v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const fx w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = fx_add(v, w);
  }
  return v;
}
// Real reflectors (float-float copies) on a float-float vector, as tri_apply_q_r.
__device__ void tri_apply_q_rx(const fx* A, const fx* tau, int n, fx* b, bool back) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  for (int s = 0; s + 1 < n; ++s) {
    const int k = back ? n - 2 - s : s;
    const fx tk = tau[k];
    if (fx_is_zero(tk)) continue;
    const fx* vk = A + (size_t)k * n;
    fx_acc acc;
    for (int i = lane; i < n; i += 32)
      if (i > k) acc.mac(vk[i], b[i]);
    const fx f = fx_mul(tk, warp_sum_x(acc.value()));
    __syncwarp();
    for (int i = lane; i < n; i += 32)
      if (i > k) b[i] = fx_sub(b[i], fx_mul(f, vk[i]));
    __syncwarp();
  }
}
// 1 / ||b|| in single precision (a scale for normalising)
__device__ __forceinline__ float inv_norm_x(const fx* b, int n) {
  const int lane = threadIdx.x & 31;
  float s = 0.f;
  for (int i = lane; i < n; i += 32) s = fmaf(b[i].hi, b[i].hi, s);
  s = warp_sum(s);
  return s > 0.f ? rsqrtf(s) : 1.f;
}

// Steps 2-4 for a real sample whose T the CTA has reduced in double precision
// (W.d, W.e; reflectors in W.A, W.tau): the brackets' single-precision rounds
// as in tri_solve_lead, then T, the reflectors and everything after them in
// float-float (overwriting the double copies in place).  Returns the number of
// refinement steps (steps_far or steps_near, as tri_solve_lead).
__device__ int tri_solve_lead_rx(const TriWs& W, const cd* G, int n, int steps_far, int steps_near,
                                 double refine_gap, TriResult& res, double& gs, double& tnorm,
                                 long long* tk) {
  const int lane = threadIdx.x & 31;
  double gmax = 0.0;
  for (int i = lane; i < n; i += 32) gmax = fmax(gmax, G[(size_t)i * n + i].re);
  gmax = warp_max(gmax);
  if (!(gmax > 0.0)) {
    for (int i = lane; i < n; i += 32) W.x[i] = mk(i == 0 ? 1.0 : 0.0, 0.0);
    __syncwarp();
    res.lam_min = res.lam_2 = res.lam_max = 0.0;
    res.near_degenerate = 1;
    gs = 1.0;
    tnorm = 0.0;
    return 0;
  }
  int ex;
  frexp(gmax, &ex);
  gs = ldexp(1.0, ex);
  double glo = 1e300, ghi = -1e300;
  for (int i = lane; i < n; i += 32) {
    const double rad = (i > 0 ? fabs(W.e[i - 1]) : 0.0) + (i + 1 < n ? fabs(W.e[i]) : 0.0);
    glo = fmin(glo, W.d[i] - rad);
    ghi = fmax(ghi, W.d[i] + rad);
    const double e2 = i + 1 < n ? W.e[i] * W.e[i] : 0.0;
    W.e2[i] = e2;
    W.df[i] = (float)W.d[i];
    W.e2f[i] = (float)e2;
  }
  glo = -warp_max(-glo);
  ghi = warp_max(ghi);
  tnorm = fmax(fabs(glo), fabs(ghi));
  glo -= 4e-13 * tnorm + 1e-300;
  ghi += 4e-13 * tnorm + 1e-300;
  __syncwarp();
  const int which[3] = {0, n > 1 ? 1 : 0, n - 1};
  Bracket br[3] = {{glo, ghi}, {glo, ghi}, {glo, ghi}};
  const double fl = 1e-5 * tnorm;
  const float tiny_f = (float)(1e-30 * fmax(tnorm, 1e-8));
  for (int round = 0; round < 12; ++round) {
    int t = -1;
    for (int m = 2; m >= 0; --m)
      if (br[m].hi - br[m].lo > fl) t = m;
    if (t < 0) break;
    multisect<true>(W, n, t, br, 3, which, tiny_f);
  }
  for (int m = 0; m < 3; ++m) {
    br[m].lo = fmax(glo, br[m].lo - 4e-6 * tnorm);
    br[m].hi = fmin(ghi, br[m].hi + 4e-6 * tnorm);
  }
  // T in float-float, in place of its double copies
  fx* dx = (fx*)W.d;
  fx* ex_ = (fx*)W.e;
  fx* e2x = (fx*)W.e2;
  for (int i = lane; i < n; i += 32) {
    const double d = W.d[i], e = W.e[i], e2 = W.e2[i];
    dx[i] = fx_of(d);
    ex_[i] = fx_of(e);
    e2x[i] = fx_of(e2);
  }
  __syncwarp();
  {
    const int m = lane % 3, end = (lane / 3) & 1;
    const double sig = end ? br[m].hi : br[m].lo;
    const int c = lane < 6 ? sturm_count_x(dx, e2x, n, fx_of(sig)) : 0;
    const bool bad = lane < 6 && (end ? c <= which[m] : c > which[m]);
    const unsigned badm = __ballot_sync(0xffffffffu, bad);
    for (int m2 = 0; m2 < 3; ++m2)
      if (badm & (0x9u << m2)) br[m2] = Bracket{glo, ghi};
  }
  const double tol_abs = 1e-13 * tnorm;
  for (int round = 0; round < 40; ++round) {
    const double w0 = br[0].hi - br[0].lo;
    if (w0 <= tol_abs || (n > 1 && br[1].lo > br[0].hi && w0 <= 1e-4 * (br[1].lo - br[0].hi)))
      break;
    multisect_x(dx, e2x, n, 0, br, 3, which);
  }
  if (n > 1) {
    for (int round = 0; round < 40; ++round) {
      const double w1 = br[1].hi - br[1].lo;
      if (w1 <= fmax(tol_abs, 1e-5 * fabs(br[1].hi))) break;
      multisect_x(dx, e2x, n, 1, br, 3, which);
    }
  }
  for (int round = 0; round < 40; ++round) {
    const double w2 = br[2].hi - br[2].lo;
    if (w2 <= fmax(tol_abs, 1e-7 * fabs(br[2].hi))) break;
    multisect_x(dx, e2x, n, 2, br, 3, which);
  }
  if (tk && lane == 0) tk[2] = clock64();
  const double lam0 = 0.5 * (br[0].lo + br[0].hi);
  const double lam1 = n > 1 ? 0.5 * (br[1].lo + br[1].hi) : lam0;
  const double lamn = 0.5 * (br[2].lo + br[2].hi);
  // the reflectors in float-float, in place (rows k, entries i > k)
  fx* Ax = (fx*)W.A;
  fx* taux = (fx*)W.tau;
  {
    const double* A = (const double*)W.A;
    const double* tau = (const double*)W.tau;
    for (int idx = lane; idx < n * n; idx += 32) {
      const double v = A[idx];
      if (idx % n > idx / n) Ax[idx] = fx_of(v);
    }
    for (int i = lane; i < n; i += 32) {
      const double v = tau[i];
      taux[i] = fx_of(v);
    }
    __syncwarp();
  }
  // 3. inverse iteration (three steps) from a fixed start vector; 4. x = Q y
  fx* u0 = (fx*)W.u0;
  fx* u1 = (fx*)W.u1;
  fx* u2 = (fx*)W.u2;
  fx* lm = (fx*)W.lm;
  tri_lu_x(dx, ex_, u0, u1, u2, lm, W.piv, n, fx_of(lam0), (float)(1e-14 * tnorm));
  fx* y = (fx*)W.z;
  for (int i = lane; i < n; i += 32) y[i] = fx{1.0f + 0.25f * (float)((i * 7) % 5), 0.f};
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    tri_solve_x(u0, u1, u2, lm, W.piv, n, y);
    __syncwarp();
    const float sc = inv_norm_x(y, n);
    for (int i = lane; i < n; i += 32) y[i] = fx_scale(y[i], sc);
    __syncwarp();
  }
  tri_apply_q_rx(Ax, taux, n, y, true);
  for (int i = lane; i < n; i += 32) W.x[i] = mk(fx_val(y[i]), 0.0);
  __syncwarp();
  const double sc = rsqrt_safe(tri_norm2(W.x, n));
  for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
  __syncwarp();
  if (tk && lane == 0) tk[3] = clock64();
  res.lam_min = gs * lam0;
  res.lam_2 = gs * lam1;
  res.lam_max = gs * lamn;
  res.near_degenerate = n > 1 && (lam1 - lam0) <= 1e-4 * lamn ? 1 : 0;
  const bool near = n > 1 && (lam1 - lam0) <= refine_gap * lamn;
  return near ? steps_near : steps_far;
}

// The Olsen step of tri_olsen_real_block with tri_solve_lead_rx's float-float
// T and reflectors (three warps: Q^T r, Q^T x with the factorisation, then
// the two solves; warp 0 finishes).
__device__ void tri_olsen_real_block_x(const TriWs& W, int n, double gs, double tnorm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const fx* Ax = (const fx*)W.A;
  const fx* taux = (const fx*)W.tau;
  const fx* dx = (const fx*)W.d;
  const fx* ex_ = (const fx*)W.e;
  fx* u0 = (fx*)W.u0;
  fx* u1 = (fx*)W.u1;
  fx* u2 = (fx*)W.u2;
  fx* lm = (fx*)W.lm;
  const double igs = 1.0 / gs;
  fx* ru = (fx*)W.q;        // Q^T r, then u
  fx* yt = ru + n;          // Q^T x
  fx* zt = (fx*)W.z;        // z, then the correction
  double th = 0.0;
  for (int i = lane; i < n; i += 32) th = fma(W.x[i].re, W.r[i].re, th);
  const double theta = warp_sum(th);
  if (warp == 0) {
    for (int i = lane; i < n; i += 32) ru[i] = fx_of(W.r[i].re - theta * W.x[i].re);
    tri_apply_q_rx(Ax, taux, n, ru, false);
  } else if (warp == 1) {
    for (int i = lane; i < n; i += 32) yt[i] = fx_of(W.x[i].re);
    tri_apply_q_rx(Ax, taux, n, yt, false);
    for (int i = lane; i < n; i += 32) zt[i] = yt[i];
    __syncwarp();
  } else if (warp == 2) {
    tri_lu_x(dx, ex_, u0, u1, u2, lm, W.piv, n, fx_of(theta * igs), (float)(1e-14 * tnorm));
  }
  __syncthreads();
  if (warp == 0) tri_solve_x(u0, u1, u2, lm, W.piv, n, ru);
  else if (warp == 1) tri_solve_x(u0, u1, u2, lm, W.piv, n, zt);
  __syncthreads();
  if (warp == 0) {
    fx_acc nu, de;
    for (int i = lane; i < n; i += 32) {
      nu.mac(yt[i], ru[i]);
      de.mac(yt[i], zt[i]);
    }
    const fx nuv = warp_sum_x(nu.value()), dev = warp_sum_x(de.value());
    const fx ep = fx_is_zero(dev) ? fx{0.f, 0.f} : fx_div(nuv, dev);
    const float ig = (float)igs;   // a power of two: exact
    for (int i = lane; i < n; i += 32) zt[i] = fx_scale(fx_sub(fx_mul(ep, zt[i]), ru[i]), ig);
    tri_apply_q_rx(Ax, taux, n, zt, true);
    for (int i = lane; i < n; i += 32) W.x[i] = mk(W.x[i].re + fx_val(zt[i]), 0.0);
    __syncwarp();
    const double sc = rsqrt_safe(tri_norm2(W.x, n));
    for (int i = lane; i < n; i += 32) W.x[i] = sc * W.x[i];
    __syncwarp();
  }
  __syncthreads();
}


// G: the n x n matrix (row-major, global or shared memory).  Result in W.x
// (unit norm).  Steps of the exact-operator refinement: `steps_far` when the
// two smallest eigenvalues are more than refine_gap * lam_max apart,
// `steps_near` otherwise.  apply(x, out): out = (exact operator) x, by the
// whole CTA (BLOCK) or by the calling warp.  BLOCK: every thread of the CTA
// calls; warp 0 does all but the operator; the result is valid in warp 0.
// single: complex matrices try the single-precision solve first.
template <typename E, bool BLOCK, class Apply>
__device__ TriResult tri_smallest(const TriWs& W, const cd* G, int n, int steps_far,
                                  int steps_near, double refine_gap, const Apply& apply,
                                  long long* tk = nullptr, bool single = false,
                                  const cfx* Gx = nullptr, bool ffr = false) {
  const int lane = threadIdx.x & 31;
  const bool lead = !BLOCK || threadIdx.x < 32;
  TriResult res = {};
  double gs = 1.0, tnorm = 0.0;
  int steps = 0;
  bool pre = false;
  if (BLOCK && !single) {
    // the CTA reduces G * 2^-ex together (ex from the largest diagonal entry)
    double gmax = 0.0;
    for (int i = lane; i < n; i += 32) gmax = fmax(gmax, G[(size_t)i * n + i].re);
    gmax = warp_max(gmax);
    if (gmax > 0.0) {
      int ex;
      frexp(gmax, &ex);
      const double igs = ldexp(1.0, -ex);
      E* A = (E*)W.A;
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        if constexpr (sizeof(E) == sizeof(double)) A[idx] = mk_e<E, double>(G[idx].re * igs, 0.0);
        else A[idx] = mk_e<E, double>(G[idx].re * igs, G[idx].im * igs);
      }
      __syncthreads();
      if (tk && threadIdx.x == 0) tk[0] = clock64();
      tri_reduce_block<E>(A, (E*)W.tau, (E*)W.w, W.d, W.e, n, (E*)W.part);
      if (tk && threadIdx.x == 0) tk[1] = clock64();
      pre = true;
    }
  }
  bool pre_sp = false;
  if constexpr (BLOCK && sizeof(E) == sizeof(cd)) {
    if (single && n > 2) {
      // the CTA reduces the single-precision copy G * 2^-ex together; the
      // lead warp goes on from T (a double-precision solve, if it follows,
      // reduces G again on its own)
      double gmax = 0.0;
      for (int i = lane; i < n; i += 32) gmax = fmax(gmax, G[(size_t)i * n + i].re);
      gmax = warp_max(gmax);
      if (gmax > 0.0) {
        int ex;
        frexp(gmax, &ex);
        const float igsf = (float)ldexp(1.0, -ex);
        cf* A = (cf*)W.A;
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x)
          A[idx] = mk((float)G[idx].re * igsf, (float)G[idx].im * igsf);
        __syncthreads();
        if (tk && threadIdx.x == 0) tk[0] = clock64();
        tri_reduce_block<cf>(A, (cf*)W.tau, (cf*)W.w, W.df, (float*)W.e, n, (cf*)W.part);
        if (tk && threadIdx.x == 0) tk[1] = clock64();
        pre_sp = true;
      }
    }
  }
  __shared__ double gt[2];   // block mode: the lead's scale and ||T|| for the other warps
  if (lead) {
    if (single && n > 2 && tri_solve_lead_sp(W, G, n, res, gs, tnorm, tk, pre_sp, Gx))
      steps = 0;
    else if (ffr && pre)   // real sample, mixed path: float-float steps 2-5
      steps = tri_solve_lead_rx(W, G, n, steps_far, steps_near, refine_gap, res, gs, tnorm, tk);
    else
      steps = tri_solve_lead<E>(W, G, n, steps_far, steps_near, refine_gap, res, gs, tnorm, tk, pre);
    if (BLOCK && lane == 0) {
      W.iv[0] = steps;
      gt[0] = gs;
      gt[1] = tnorm;
    }
  }
  if (BLOCK) {
    __syncthreads();
    steps = W.iv[0];
    gs = gt[0];
    tnorm = gt[1];
  }
  // real samples on a CTA of three or more warps: the step's chains in parallel
  const bool par = BLOCK && sizeof(E) == sizeof(double) && blockDim.x >= 96;
  for (int it = 0; it < steps; ++it) {
    apply(W.x, W.r);
    team_sync<BLOCK>();
    if (tk && lead && lane == 0) tk[6] = clock64();   // end of the last step's apply
    if constexpr (BLOCK && sizeof(E) == sizeof(double)) {
      if (par) {
        if (ffr && pre) tri_olsen_real_block_x(W, n, gs, tnorm);
        else tri_olsen_real_block(W, n, gs, tnorm);
        continue;
      }
    }
    if (lead) tri_olsen<E>(W, n, gs, tnorm);
    team_sync<BLOCK>();
  }
  if (tk && lead && lane == 0) tk[4] = clock64();
  if (lead) {
    // theta = x^H G x
    cd th = mk(0.0, 0.0);
    cfx* xx = (cfx*)W.part;
    if (Gx) {
      for (int i = lane; i < n; i += 32) xx[i] = cfx_of(W.x[i]);
      __syncwarp();
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int i = lane + 32 * c;
      if (i < n) {
        cd gx = mk(0.0, 0.0);
        if (Gx) {
          cfx_acc acc;
          for (int j = 0; j < n; ++j) acc.macc(Gx[(size_t)j * n + i], xx[j]);
          gx = cfx_val(acc.value());
        } else {
          for (int j = 0; j < n; ++j) cfmac(gx, G[(size_t)j * n + i], W.x[j]);   // (G x)_i
        }
        cfmac(th, W.x[i], gx);
      }
    }
    res.theta = warp_sum(th.re);
  }
  if (tk && lead && lane == 0) tk[5] = clock64();
  return res;
}
