// A8: learned kernel proposal -- forward, backward and AdamW kernels.
//
// The network sees both blurred frames: the luma (channel mean) of each,
// area-downsampled to 256 x 256, then
//   conv 3x3 s2 p1 (2 -> 32) + ReLU, conv 3x3 s2 p1 (32 -> 32) + ReLU,
//   conv 3x3 s4 p1 (32 -> 32) + ReLU, conv 2x2 s1 p0 (32 -> 2),
//   softmax over each output channel's 15 x 15 logits -> K1, K2.
// Activations are stored as bfloat16 and weights kept as float32 master
// copies.  The forward convolutions run on the tensor cores (tcgen05, BF16
// operands with the weights rounded to BF16, FP32 accumulation in tensor
// memory) as implicit GEMMs over 128 output positions per CTA; the backward
// pass (training only) stays on the FP32 units with the float32 weights, a
// thread per output and weight gradients reduced in a fixed order
// (deterministic).  Training minimises the mean squared error of both
// kernels with AdamW (decoupled weight decay).
#include <cuda_bf16.h>
#include <cstdio>
#include <cstring>
#include <vector>
#include "cbp_common.cuh"
#include "cbp_internal.h"
#include "cbp_serve.h"
#include "cbp_tc.cuh"

namespace cbp {

namespace {

using bf16 = __nv_bfloat16;

struct Layer {
  int cin, cout, k, s, p, hin, hout, woff, boff, relu;
};

__host__ __device__ inline Layer cnn_layer(int i) {
  switch (i) {
    case 0: return {2, 32, 3, 2, 1, kCnnSide, kCnnSide / 2, 0, 576, 1};
    case 1: return {32, 32, 3, 2, 1, kCnnSide / 2, kCnnSide / 4, 608, 9824, 1};
    case 2: return {32, 32, 3, 4, 1, kCnnSide / 4, kCnnSide / 16, 9856, 19072, 1};
    default: return {32, 2, 2, 1, 0, kCnnSide / 16, kCnnT, 19104, 19360, 0};
  }
}

constexpr int kCnnThreads = 256;
constexpr int kT2 = kCnnT * kCnnT;

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;
constexpr uint32_t kTcCols = 32;   // tensor-memory columns per CTA (>= N, a power of two >= 32)
template <int CIN, int KS, int N>
struct ConvTc {
  static constexpr int kK = KS * KS * CIN;
  static constexpr int kKpad = (kK + 15) / 16 * 16;
  static constexpr int kGroups = kKpad / 8;                 // K-groups of 8
  static constexpr uint32_t kAGroup = kTcM * 16;            // bytes per K-group of A
  static constexpr uint32_t kBGroup = N * 16;               // bytes per K-group of B
  static constexpr int kBBytes = kKpad * N * 2;
  static constexpr int kABytes = kKpad * kTcM * 2;
  static constexpr int kSmem = kBBytes + kABytes;
};
// The four layers' shapes: (CIN, KS, N).
using Tc0 = ConvTc<2, 3, 32>;
using Tc1 = ConvTc<32, 3, 32>;
using Tc2 = ConvTc<32, 3, 32>;
using Tc3 = ConvTc<32, 2, 16>;
// Byte offsets of the layers' B images in the weight-image buffer.
__host__ __device__ constexpr int tc_img_offset(int li) {
  return (li > 0 ? Tc0::kBBytes : 0) + (li > 1 ? Tc1::kBBytes : 0) + (li > 2 ? Tc2::kBBytes : 0) +
         (li > 3 ? Tc3::kBBytes : 0);
}

// Workspace layout (byte offsets) for n pairs.
struct CnnWs {
  size_t x0, a1, a2, a3, z4, k, wimg, dz4, dz3, dz2, dz1, grad, lossp, total;
};
size_t al(size_t x) { return (x + 255) & ~size_t(255); }
CnnWs cnn_ws_layout(int n, bool train) {
  CnnWs L{};
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t r = o;
    o += al(b);
    return r;
  };
  const size_t N = n;
  L.x0 = take(N * 2 * kCnnSide * kCnnSide * sizeof(bf16));
  L.a1 = take(N * 32 * (kCnnSide / 2) * (kCnnSide / 2) * sizeof(bf16));
  L.a2 = take(N * 32 * (kCnnSide / 4) * (kCnnSide / 4) * sizeof(bf16));
  L.a3 = take(N * 32 * (kCnnSide / 16) * (kCnnSide / 16) * sizeof(bf16));
  L.z4 = take(N * 2 * kT2 * 4);
  L.k = take(N * 2 * kT2 * 4);
  L.wimg = take(tc_img_offset(4));
  if (train) {
    L.dz4 = take(N * 2 * kT2 * 4);
    L.dz3 = take(N * 32 * (kCnnSide / 16) * (kCnnSide / 16) * 4);
    L.dz2 = take(N * 32 * (kCnnSide / 4) * (kCnnSide / 4) * 4);
    L.dz1 = take(N * 32 * (kCnnSide / 2) * (kCnnSide / 2) * 4);
    L.grad = take((size_t)kCnnParams * 4);
    L.lossp = take(N * 2 * 4);
  }
  L.total = o;
  return L;
}

// Area resampling of the luma of frame z of pair f to kCnnSide x kCnnSide:
// output cell (y, x) averages the input over [y fy, (y+1) fy) x [x fx, (x+1) fx),
// partial input cells weighted by their overlap.
__global__ void __launch_bounds__(kCnnThreads) k_cnn_input(FrameDesc f1, FrameDesc f2, bf16* x0) {
  const int z = blockIdx.y, f = blockIdx.z;
  const FrameDesc& fr = z ? f2 : f1;
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= kCnnSide * kCnnSide) return;
  const int y = o / kCnnSide, x = o % kCnnSide;
  // cell bounds in exact integer arithmetic: [y h / S, (y + 1) h / S)
  const int r0 = (int)(((int64_t)y * fr.h) / kCnnSide);
  const int r1 = min(fr.h, (int)(((int64_t)(y + 1) * fr.h + kCnnSide - 1) / kCnnSide));
  const int c0 = (int)(((int64_t)x * fr.w) / kCnnSide);
  const int c1 = min(fr.w, (int)(((int64_t)(x + 1) * fr.w + kCnnSide - 1) / kCnnSide));
  // overlaps in units of 1/S input cells: [y h, (y+1) h) against [r S, (r+1) S)
  const int ya = y * fr.h, yb = (y + 1) * fr.h, xa = x * fr.w, xb = (x + 1) * fr.w;
  const void* base = frame_base(fr, f);
  float acc = 0.f;
  for (int r = r0; r < r1; ++r) {
    const int wy = min(yb, (r + 1) * kCnnSide) - max(ya, r * kCnnSide);
    const int64_t rb = (int64_t)r * fr.rs;
    float row = 0.f;
    for (int c = c0; c < c1; ++c) {
      const int wx = min(xb, (c + 1) * kCnnSide) - max(xa, c * kCnnSide);
      float v = 0.f;
      for (int ch = 0; ch < fr.c; ++ch) v += ld_frame<float>(base, (int64_t)ch * fr.cs + rb + c, fr.f64);
      row = fmaf((float)wx, v, row);
    }
    acc = fmaf((float)wy, row, acc);
  }
  // weights were in 1/S units of an input cell; the cell area is h w / S^2
  const float norm = 1.0f / ((float)fr.h * (float)fr.w * (float)fr.c);
  x0[((int64_t)f * 2 + z) * kCnnSide * kCnnSide + o] = __float2bfloat16(acc * norm);
}

// The same resampling with one CTA per output row: the input rows of the row's
// cells are read once, coalesced (a thread per input column), weighted by
// their overlaps and summed over rows and channels into a shared column
// profile; each output cell then sums its columns' profile with the column
// overlaps.  Widths up to kCnnMaxW.
constexpr int kCnnMaxW = 8192;
constexpr int kCnnColsPT = 8;
template <typename In>
__device__ __forceinline__ void cnn_profile_cols(const In* base, const FrameDesc& fr, int r0, int r1,
                                                 int ya, int yb, float* prof) {
  float col[kCnnColsPT], v[kCnnColsPT];
#pragma unroll
  for (int j = 0; j < kCnnColsPT; ++j) col[j] = 0.f;
  for (int r = r0; r < r1; ++r) {
    const int wy = min(yb, (r + 1) * kCnnSide) - max(ya, r * kCnnSide);
#pragma unroll
    for (int j = 0; j < kCnnColsPT; ++j) v[j] = 0.f;
    for (int ch = 0; ch < fr.c; ++ch) {
      const In* row = base + (int64_t)ch * fr.cs + (int64_t)r * fr.rs + threadIdx.x;
#pragma unroll
      for (int j = 0; j < kCnnColsPT; ++j)
        if ((int)threadIdx.x + j * kCnnThreads < fr.w) v[j] += (float)__ldg(row + j * kCnnThreads);
    }
#pragma unroll
    for (int j = 0; j < kCnnColsPT; ++j) col[j] = fmaf((float)wy, v[j], col[j]);
  }
#pragma unroll
  for (int j = 0; j < kCnnColsPT; ++j) {
    const int c = threadIdx.x + j * kCnnThreads;
    if (c < fr.w) prof[c] = col[j];
  }
}

__global__ void __launch_bounds__(kCnnThreads) k_cnn_input_rows(FrameDesc f1, FrameDesc f2, bf16* x0) {
  __shared__ float prof[kCnnMaxW];
  const int y = blockIdx.x, z = blockIdx.y, f = blockIdx.z;
  const FrameDesc& fr = z ? f2 : f1;
  const int r0 = (int)(((int64_t)y * fr.h) / kCnnSide);
  const int r1 = min(fr.h, (int)(((int64_t)(y + 1) * fr.h + kCnnSide - 1) / kCnnSide));
  const int ya = y * fr.h, yb = (y + 1) * fr.h;
  const void* base = frame_base(fr, f);
  if (fr.w <= kCnnColsPT * kCnnThreads) {
    // kCnnColsPT columns per thread: their loads of one (row, channel) are in
    // flight together
    if (fr.f64) cnn_profile_cols<double>((const double*)base, fr, r0, r1, ya, yb, prof);
    else cnn_profile_cols<float>((const float*)base, fr, r0, r1, ya, yb, prof);
  } else {
    for (int c = threadIdx.x; c < fr.w; c += blockDim.x) {
      float col = 0.f;
      for (int r = r0; r < r1; ++r) {
        const int wy = min(yb, (r + 1) * kCnnSide) - max(ya, r * kCnnSide);
        const int64_t rb = (int64_t)r * fr.rs + c;
        float v = 0.f;
        for (int ch = 0; ch < fr.c; ++ch) v += ld_frame<float>(base, (int64_t)ch * fr.cs + rb, fr.f64);
        col = fmaf((float)wy, v, col);
      }
      prof[c] = col;
    }
  }
  __syncthreads();
  const float norm = 1.0f / ((float)fr.h * (float)fr.w * (float)fr.c);
  for (int x = threadIdx.x; x < kCnnSide; x += blockDim.x) {
    const int c0 = (int)(((int64_t)x * fr.w) / kCnnSide);
    const int c1 = min(fr.w, (int)(((int64_t)(x + 1) * fr.w + kCnnSide - 1) / kCnnSide));
    const int xa = x * fr.w, xb = (x + 1) * fr.w;
    float acc = 0.f;
    for (int c = c0; c < c1; ++c) {
      const int wx = min(xb, (c + 1) * kCnnSide) - max(xa, c * kCnnSide);
      acc = fmaf((float)wx, prof[c], acc);
    }
    x0[((int64_t)f * 2 + z) * kCnnSide * kCnnSide + (int64_t)y * kCnnSide + x] =
        __float2bfloat16(acc * norm);
  }
}

template <typename TO> __device__ __forceinline__ TO to_out(float v);
template <> __device__ __forceinline__ bf16 to_out<bf16>(float v) { return __float2bfloat16(v); }
template <> __device__ __forceinline__ float to_out<float>(float v) { return v; }

// Convolutions on the tensor cores (tcgen05), as implicit GEMMs:
//   y[n][co][o] = b[co] + sum_k A[o][k] B[co][k],
// o an output position, k = (u KS + v) CIN + ci a tap and an input channel,
// A[o][k] = x[n][ci][oy s - p + u][ox s - p + v] (zero outside x) and
// B[co][k] = w[co][ci][u][v] rounded to BF16.  A CTA takes 128 consecutive
// output positions (tcgen05's M) and all output channels (N = 32; 16 for the
// two-channel head, its rows 2..15 zero): its eight warps gather A from the
// BF16 activations into shared memory, one thread issues the K / 16 MMAs into
// an FP32 accumulator in tensor memory, and each warp reads back 16 channels
// of 32 positions for the epilogue (bias, ReLU, store).  K is padded with
// zeros to a multiple of 16.
constexpr int kTcWaitLimit = 1 << 20;

// B images of all four layers (BF16, the shared-memory layout of
// cbp_tc.cuh), one layer per blockIdx.y; rows co >= cout and columns
// k >= KS^2 CIN are zero.
template <int CIN, int KS, int N>
__device__ void conv_w_image(const float* prm, const Layer& L, uint8_t* img) {
  using C = ConvTc<CIN, KS, N>;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * C::kKpad; i += gridDim.x * blockDim.x) {
    const int co = i / C::kKpad, k = i - co * C::kKpad;
    float w = 0.f;
    if (co < L.cout && k < C::kK) {
      const int tap = k / CIN, ci = k - tap * CIN;
      w = prm[L.woff + (co * CIN + ci) * KS * KS + tap];
    }
    *(bf16*)(img + tc::kmajor_offset(N, co, k)) = __float2bfloat16(w);
  }
}
__global__ void k_conv_w_images(const float* prm, uint8_t* img) {
  switch (blockIdx.y) {
    case 0: conv_w_image<2, 3, 32>(prm, cnn_layer(0), img + tc_img_offset(0)); break;
    case 1: conv_w_image<32, 3, 32>(prm, cnn_layer(1), img + tc_img_offset(1)); break;
    case 2: conv_w_image<32, 3, 32>(prm, cnn_layer(2), img + tc_img_offset(2)); break;
    default: conv_w_image<32, 2, 16>(prm, cnn_layer(3), img + tc_img_offset(3)); break;
  }
}

template <int CIN, int KS, int N, typename TO>
__global__ void __launch_bounds__(kTcThreads) k_conv_tc(const bf16* __restrict__ x,
                                                         const uint8_t* __restrict__ wimg,
                                                         const float* __restrict__ prm, TO* __restrict__ y,
                                                         Layer L, int* err) {
  using C = ConvTc<CIN, KS, N>;
  extern __shared__ __align__(128) uint8_t tsm[];
  __shared__ uint64_t done;
  __shared__ uint32_t tslot;
  uint8_t* sB = tsm;
  uint8_t* sA = tsm + C::kBBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = blockIdx.y, npos = L.hout * L.hout, m0 = blockIdx.x * kTcM;

  if (warp == 0) tc::tmem_alloc(&tslot, kTcCols);
  if (tid == 0) tc::bar_init(&done, 1);
  for (int i = tid; i < C::kBBytes / 16; i += kTcThreads)
    ((uint4*)sB)[i] = __ldg((const uint4*)wimg + i);
  // A: thread-chunk (m, g) holds k = 8g .. 8g + 7 of position m0 + m; the
  // warp's 32 chunks are 32 consecutive positions, stored as 512 contiguous bytes
  const unsigned short* xs = reinterpret_cast<const unsigned short*>(x) + (int64_t)n * CIN * L.hin * L.hin;
  const int64_t plane = (int64_t)L.hin * L.hin;
#pragma unroll 2
  for (int c = tid; c < kTcM * C::kGroups; c += kTcThreads) {
    const int m = c & (kTcM - 1), g = c / kTcM;
    const int o = m0 + m;
    uint32_t q[4] = {0u, 0u, 0u, 0u};
    if (o < npos) {
      const int oy = o / L.hout, ox = o - oy * L.hout;
      const int iy0 = oy * L.s - L.p, ix0 = ox * L.s - L.p;
      if constexpr (CIN % 8 == 0) {   // the group is 8 channels of one tap
        const int tap = g / (CIN / 8), ci0 = (g - tap * (CIN / 8)) * 8;
        const int u = tap / KS, v = tap - u * KS;
        const int iy = iy0 + u, ix = ix0 + v;
        if (tap < KS * KS && iy >= 0 && iy < L.hin && ix >= 0 && ix < L.hin) {
          const unsigned short* px = xs + ci0 * plane + (int64_t)iy * L.hin + ix;
#pragma unroll
          for (int e = 0; e < 8; ++e) q[e >> 1] |= (uint32_t)__ldg(px + e * plane) << (16 * (e & 1));
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = g * 8 + e;
          const int tap = k / CIN, ci = k - tap * CIN;
          const int u = tap / KS, v = tap - u * KS;
          const int iy = iy0 + u, ix = ix0 + v;
          if (tap < KS * KS && iy >= 0 && iy < L.hin && ix >= 0 && ix < L.hin)
            q[e >> 1] |= (uint32_t)__ldg(xs + ci * plane + (int64_t)iy * L.hin + ix) << (16 * (e & 1));
        }
      }
    }
    *(uint4*)(sA + tc::kmajor_offset(kTcM, m, 8 * g)) = make_uint4(q[0], q[1], q[2], q[3]);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint32_t a0 = tc::saddr(sA), b0 = tc::saddr(sB);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, N);
#pragma unroll 1
    for (int s = 0; s < C::kKpad / 16; ++s)
      tc::mma_bf16(tmem, tc::sdesc(a0 + 2 * s * C::kAGroup, C::kAGroup, 128),
                   tc::sdesc(b0 + 2 * s * C::kBGroup, C::kBGroup, 128), idesc, s > 0);
    tc::mma_commit(&done);
  }
  const bool arrived = tc::bar_wait(&done, 0, kTcWaitLimit);
  const bool late = __syncthreads_or(!arrived);
  if (late) {
    // the MMAs did not complete in time: report it, wait once more (bounded)
    // and leave NaN outputs behind
    if (tid == 0 && err) atomicOr(err, 1);
    if (!arrived) tc::bar_wait(&done, 0, kTcWaitLimit);
  }
  tc::fence_after_sync();
  const int quarter = warp & 3, half = warp >> 2;
  if (half * 16 < N) {
    float v[16];
    if (!late) {
      tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + half * 16, v);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = __int_as_float(0x7fc00000);
    }
    const int o = m0 + quarter * 32 + lane;
    if (o < npos) {
      TO* yo = y + (int64_t)n * L.cout * npos + o;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int co = half * 16 + j;
        if (co < L.cout) {
          float a = v[j] + __ldg(prm + L.boff + co);
          if (L.relu) a = fmaxf(a, 0.f);
          yo[(int64_t)co * npos] = to_out<TO>(a);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, kTcCols);
  }
}

template <int CIN, int KS, int N, typename TO>
void run_conv_tc(const bf16* x, const uint8_t* img, const float* prm, TO* y, int li, int n, int* err,
                 cudaStream_t st) {
  using C = ConvTc<CIN, KS, N>;
  const Layer L = cnn_layer(li);
  const int npos = L.hout * L.hout;
  auto kfn = k_conv_tc<CIN, KS, N, TO>;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  kfn<<<dim3((npos + kTcM - 1) / kTcM, n), kTcThreads, C::kSmem, st>>>(x, img + tc_img_offset(li), prm, y, L, err);
}

// Softmax of each (pair, head) over its 225 logits; with targets, the loss
// terms and the logits' gradient of L = sum (K - K_true)^2 / (n 2 225).
__global__ void k_softmax(const float* z, float* K, const float* kt, float* dz, float* lossp, int n) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n * 2) return;
  const float* zz = z + (int64_t)w * kT2;
  float m = -INFINITY;
  for (int j = lane; j < kT2; j += 32) m = fmaxf(m, zz[j]);
  m = warp_max(m);
  float s = 0.f;
  for (int j = lane; j < kT2; j += 32) s += expf(zz[j] - m);
  s = warp_sum(s);
  const float inv = 1.f / s;
  for (int j = lane; j < kT2; j += 32) K[(int64_t)w * kT2 + j] = expf(zz[j] - m) * inv;
  if (!kt) return;
  __syncwarp();
  const float scale = 2.f / (float)(n * 2 * kT2);
  float gp = 0.f, l = 0.f;
  for (int j = lane; j < kT2; j += 32) {
    const float p = K[(int64_t)w * kT2 + j], d = p - kt[(int64_t)w * kT2 + j];
    gp += scale * d * p;
    l += d * d;
  }
  gp = warp_sum(gp);
  l = warp_sum(l);
  for (int j = lane; j < kT2; j += 32) {
    const float p = K[(int64_t)w * kT2 + j], d = p - kt[(int64_t)w * kT2 + j];
    dz[(int64_t)w * kT2 + j] = p * (scale * d - gp);
  }
  if (lane == 0) lossp[w] = l;
}

__global__ void k_loss_sum(const float* lossp, int m, float denom, float* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < m; ++i) s += lossp[i];
    out[0] = s / denom;
  }
}

// dx[n][ci][iy][ix] = sum_{co,u,v: iy = oy s - p + u, ix = ox s - p + v} w[co][ci][u][v] dy[n][co][oy][ox],
// times the ReLU mask of the layer input (x > 0): the gradient of the
// previous layer's pre-activation.
__global__ void __launch_bounds__(kCnnThreads)
k_conv_bwd_data(const float* dy, const float* prm, const bf16* xact, float* dx, Layer L) {
  extern __shared__ float ws[];
  const int ci = blockIdx.y, n = blockIdx.z;
  const int kk = L.k * L.k;
  for (int i = threadIdx.x; i < L.cout * kk; i += blockDim.x) {
    const int co = i / kk, uv = i % kk;
    ws[i] = prm[L.woff + (co * L.cin + ci) * kk + uv];
  }
  __syncthreads();
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= L.hin * L.hin) return;
  const int iy = o / L.hin, ix = o % L.hin;
  const int64_t xi = ((int64_t)n * L.cin + ci) * L.hin * L.hin + o;
  if (!(__bfloat162float(xact[xi]) > 0.f)) {
    dx[xi] = 0.f;
    return;
  }
  float acc = 0.f;
  for (int u = 0; u < L.k; ++u) {
    const int ty = iy + L.p - u;
    if (ty < 0 || ty % L.s) continue;
    const int oy = ty / L.s;
    if (oy >= L.hout) continue;
    for (int v = 0; v < L.k; ++v) {
      const int tx = ix + L.p - v;
      if (tx < 0 || tx % L.s) continue;
      const int ox = tx / L.s;
      if (ox >= L.hout) continue;
      for (int co = 0; co < L.cout; ++co)
        acc = fmaf(ws[co * kk + u * L.k + v],
                   dy[(((int64_t)n * L.cout + co) * L.hout + oy) * L.hout + ox], acc);
    }
  }
  dx[xi] = acc;
}

// Weight and bias gradients of one (co, ci) pair: sum over pairs and output
// positions, block-wide tree reduction in a fixed order.
__global__ void __launch_bounds__(kCnnThreads)
k_conv_bwd_w(const float* dy, const bf16* x, float* grad, Layer L, int n) {
  __shared__ float red[10][kCnnThreads];
  const int ci = blockIdx.x, co = blockIdx.y;
  const int kk = L.k * L.k, hw = L.hout * L.hout;
  float acc[10];
#pragma unroll
  for (int j = 0; j < 10; ++j) acc[j] = 0.f;
  for (int64_t q = threadIdx.x; q < (int64_t)n * hw; q += blockDim.x) {
    const int nn = (int)(q / hw), o = (int)(q % hw);
    const int oy = o / L.hout, ox = o % L.hout;
    const float g = dy[((int64_t)nn * L.cout + co) * hw + o];
    const bf16* xc = x + ((int64_t)nn * L.cin + ci) * L.hin * L.hin;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (u >= L.k) break;
      const int iy = oy * L.s - L.p + u;
#pragma unroll
      for (int v = 0; v < 3; ++v) {
        if (v >= L.k) break;
        const int ix = ox * L.s - L.p + v;
        if (iy >= 0 && iy < L.hin && ix >= 0 && ix < L.hin)
          acc[u * 3 + v] = fmaf(g, __bfloat162float(xc[iy * L.hin + ix]), acc[u * 3 + v]);
      }
    }
    acc[9] += g;
  }
#pragma unroll
  for (int j = 0; j < 10; ++j) red[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
#pragma unroll
      for (int j = 0; j < 10; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < kk) {
    const int u = threadIdx.x / L.k, v = threadIdx.x % L.k;
    grad[L.woff + (co * L.cin + ci) * kk + threadIdx.x] = red[u * 3 + v][0];
  }
  if (ci == 0 && threadIdx.x == 0) grad[L.boff + co] = red[9][0];
}

// AdamW (Loshchilov & Hutter): m, v moments, bias-corrected step, decoupled
// weight decay.
__global__ void k_adamw(float* p, const float* g, float* m, float* v, int count, cbp_adamw hp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = hp.beta1 * m[i] + (1.f - hp.beta1) * gi;
  const float vi = hp.beta2 * v[i] + (1.f - hp.beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(hp.beta1, (float)hp.step));
  const float vh = vi / (1.f - powf(hp.beta2, (float)hp.step));
  p[i] -= hp.lr * mh / (sqrtf(vh) + hp.eps) + hp.lr * hp.weight_decay * p[i];
}

__global__ void k_bf16_to_f32(const bf16* a, float* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __bfloat162float(a[i]);
}

// Proposals into the double kernel buffer [n][t1^2 + t2^2] of the estimation
// path (K1 first, then K2).
__global__ void k_cnn_to_kd(const float* K, int n, double* kd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * 2 * kT2) return;
  kd[i] = (double)K[i];
}

// Layer li of the network on the tensor cores; wimg holds the B images
// written by k_conv_w_images for the same parameters.
void launch_conv_fwd(const bf16* x, const uint8_t* wimg, const float* prm, void* y, int li, int n,
                     int* err, cudaStream_t st) {
  switch (li) {
    case 0: run_conv_tc<2, 3, 32, bf16>(x, wimg, prm, (bf16*)y, 0, n, err, st); break;
    case 1: run_conv_tc<32, 3, 32, bf16>(x, wimg, prm, (bf16*)y, 1, n, err, st); break;
    case 2: run_conv_tc<32, 3, 32, bf16>(x, wimg, prm, (bf16*)y, 2, n, err, st); break;
    default: run_conv_tc<32, 2, 16, float>(x, wimg, prm, (float*)y, 3, n, err, st); break;
  }
}

void copy_f32(const bf16* a, float* b, int64_t n, cudaStream_t st) {
  if (b) k_bf16_to_f32<<<256, 256, 0, st>>>(a, b, n);
}

}  // namespace

size_t cnn_workspace(int n, bool train) { return cnn_ws_layout(n, train).total; }

void cnn_forward(const FrameDesc& b1, const FrameDesc& b2, int n, const float* prm, char* ws,
                 cudaStream_t st, const cbp_cnn_trace* tr, int* err) {
  const CnnWs L = cnn_ws_layout(n, false);
  bf16* x0 = (bf16*)(ws + L.x0);
  bf16* a[3] = {(bf16*)(ws + L.a1), (bf16*)(ws + L.a2), (bf16*)(ws + L.a3)};
  if (b1.w <= kCnnMaxW && b2.w <= kCnnMaxW)
    k_cnn_input_rows<<<dim3(kCnnSide, 2, n), kCnnThreads, 0, st>>>(b1, b2, x0);
  else
    k_cnn_input<<<dim3(kCnnSide * kCnnSide / kCnnThreads, 2, n), kCnnThreads, 0, st>>>(b1, b2, x0);
  uint8_t* wimg = (uint8_t*)(ws + L.wimg);
  k_conv_w_images<<<dim3(8, 4), 256, 0, st>>>(prm, wimg);
  launch_conv_fwd(x0, wimg, prm, a[0], 0, n, err, st);
  launch_conv_fwd(a[0], wimg, prm, a[1], 1, n, err, st);
  launch_conv_fwd(a[1], wimg, prm, a[2], 2, n, err, st);
  launch_conv_fwd(a[2], wimg, prm, ws + L.z4, 3, n, err, st);
  k_softmax<<<(n * 2 * 32 + 127) / 128, 128, 0, st>>>((const float*)(ws + L.z4), (float*)(ws + L.k),
                                                      nullptr, nullptr, nullptr, n);
  if (tr) {
    copy_f32(x0, tr->input, (int64_t)n * 2 * kCnnSide * kCnnSide, st);
    for (int i = 0; i < 3; ++i) {
      const Layer Ly = cnn_layer(i);
      copy_f32(a[i], tr->act[i], (int64_t)n * Ly.cout * Ly.hout * Ly.hout, st);
    }
    if (tr->logits)
      cudaMemcpyAsync(tr->logits, ws + L.z4, (size_t)n * 2 * kT2 * 4, cudaMemcpyDeviceToDevice, st);
  }
}

const float* cnn_kernels(char* ws, int n) { return (const float*)(ws + cnn_ws_layout(n, false).k); }

void cnn_to_kd(char* ws, int n, double* kd, cudaStream_t st) {
  k_cnn_to_kd<<<(n * 2 * kT2 + 255) / 256, 256, 0, st>>>(cnn_kernels(ws, n), n, kd);
}

void cnn_train_step(const FrameDesc& b1, const FrameDesc& b2, int n, const float* kt, float* prm,
                    float* m, float* v, const cbp_adamw& hp, float* loss, char* ws, cudaStream_t st,
                    const cbp_cnn_trace* tr) {
  cnn_forward(b1, b2, n, prm, ws, st, tr);
  const CnnWs L = cnn_ws_layout(n, true);
  bf16* x0 = (bf16*)(ws + L.x0);
  bf16* a[3] = {(bf16*)(ws + L.a1), (bf16*)(ws + L.a2), (bf16*)(ws + L.a3)};
  float* dz[4] = {(float*)(ws + L.dz1), (float*)(ws + L.dz2), (float*)(ws + L.dz3),
                  (float*)(ws + L.dz4)};
  float* grad = (float*)(ws + L.grad);
  k_softmax<<<(n * 2 * 32 + 127) / 128, 128, 0, st>>>((const float*)(ws + L.z4), (float*)(ws + L.k),
                                                      kt, dz[3], (float*)(ws + L.lossp), n);
  for (int li = 3; li >= 0; --li) {
    const Layer Ly = cnn_layer(li);
    const bf16* xin = li ? a[li - 1] : x0;
    k_conv_bwd_w<<<dim3(Ly.cin, Ly.cout), kCnnThreads, 0, st>>>(dz[li], xin, grad, Ly, n);
    if (li > 0) {
      dim3 g((Ly.hin * Ly.hin + kCnnThreads - 1) / kCnnThreads, Ly.cin, n);
      k_conv_bwd_data<<<g, kCnnThreads, sizeof(float) * Ly.cout * Ly.k * Ly.k, st>>>(
          dz[li], prm, a[li - 1], dz[li - 1], Ly);
    }
  }
  if (tr && tr->grad)
    cudaMemcpyAsync(tr->grad, grad, (size_t)kCnnParams * 4, cudaMemcpyDeviceToDevice, st);
  if (loss) k_loss_sum<<<1, 32, 0, st>>>((const float*)(ws + L.lossp), n * 2, (float)(n * 2 * kT2), loss);
  if (hp.lr != 0.f || hp.weight_decay != 0.f)
    k_adamw<<<(kCnnParams + 255) / 256, 256, 0, st>>>(prm, grad, m, v, kCnnParams, hp);
}

}  // namespace cbp

using cbp::Ctx;

namespace {

cbp_status cnn_frames(const cbp_frames* b1, const cbp_frames* b2, cbp::FrameDesc* d1,
                      cbp::FrameDesc* d2) {
  if (!b1 || !b2 || !b1->data || !b2->data || b1->n != b2->n || b1->n < 1 || b1->c < 1 ||
      b2->c < 1 || b1->h < 1 || b1->w < 1 || b2->h < 1 || b2->w < 1 || b1->dtype != b2->dtype)
    return CBP_ERR_INVALID_ARG;
  *d1 = cbp::frame_desc(b1, nullptr);
  *d2 = cbp::frame_desc(b2, nullptr);
  return CBP_OK;
}

}  // namespace

extern "C" {

size_t cbp_cnn_param_count(void) { return (size_t)cbp::kCnnParams; }

cbp_status cbp_cnn_forward(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                           const float* weights, float* kernels, cbp_cnn_trace* trace, void* stream) {
  if (!ctx || !kernels) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cbp::FrameDesc d1, d2;
  cbp_status s = cnn_frames(b1, b2, &d1, &d2);
  if (s != CBP_OK) return s;
  const float* w = weights ? weights : c->cnn_w;
  if (!w) return CBP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(c->api_mu);
  s = c->ensure_cnn_ws(cbp::cnn_workspace(b1->n, false), st);
  if (s != CBP_OK) return s;
  cbp::cnn_forward(d1, d2, b1->n, w, c->cnn_ws, st, trace);
  if (cudaMemcpyAsync(kernels, cbp::cnn_kernels(c->cnn_ws, b1->n),
                      (size_t)b1->n * 2 * cbp::kCnnT * cbp::kCnnT * 4, cudaMemcpyDeviceToDevice,
                      st) != cudaSuccess)
    return CBP_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

cbp_status cbp_cnn_train_step(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                              const float* k_true, float* weights, float* adam_m, float* adam_v,
                              const cbp_adamw* hp, float* loss, cbp_cnn_trace* trace, void* stream) {
  if (!ctx || !k_true || !weights || !adam_m || !adam_v || !hp || hp->step < 1)
    return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cbp::FrameDesc d1, d2;
  cbp_status s = cnn_frames(b1, b2, &d1, &d2);
  if (s != CBP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(c->api_mu);
  s = c->ensure_cnn_ws(cbp::cnn_workspace(b1->n, true), st);
  if (s != CBP_OK) return s;
  cbp::cnn_train_step(d1, d2, b1->n, k_true, weights, adam_m, adam_v, *hp, loss, c->cnn_ws, st,
                      trace);
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

cbp_status cbp_learned_load(cbp_ctx* ctx, const char* path) {
  if (!ctx || !path) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  FILE* fp = fopen(path, "rb");
  if (!fp) return CBP_ERR_INVALID_ARG;
  char magic[8];
  int32_t side = 0, count = 0;
  std::vector<float> w;
  bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, "CBPCNN1", 8) == 0 &&
            fread(&side, 4, 1, fp) == 1 && fread(&count, 4, 1, fp) == 1 &&
            side == cbp::kCnnSide && count == cbp::kCnnParams;
  if (ok) {
    w.resize(count);
    ok = fread(w.data(), 4, count, fp) == (size_t)count;
  }
  fclose(fp);
  if (!ok) return CBP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(c->api_mu);
  if (!c->cnn_w) {
    if (!c->reserve((size_t)count * 4)) return CBP_ERR_BUDGET;
    if (cudaMalloc((void**)&c->cnn_w, (size_t)count * 4) != cudaSuccess) {
      cudaGetLastError();
      c->release((size_t)count * 4);
      c->cnn_w = nullptr;
      return CBP_ERR_OOM;
    }
  }
  if (cudaMemcpy(c->cnn_w, w.data(), (size_t)count * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return CBP_ERR_CUDA;
  return CBP_OK;
}

}  // extern "C"
