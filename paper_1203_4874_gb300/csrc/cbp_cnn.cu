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
#include <algorithm>
#include <vector>
#include "cbp_common.cuh"
#include "cbp_internal.h"
#include "cbp_serve.h"
#include "cbp_nvtx.h"
#include "cbp_tc.cuh"

namespace cbp {

CBP_CHECKS_TU(kChkCnn)

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

// Shapes of the input-gradient products (transposed weights, N = CIN).
template <int CIN, int KS, int COUT>
struct ConvTcT {
  static constexpr int kK = KS * KS * COUT;
  static constexpr int kKpad = (kK + 15) / 16 * 16;
  static constexpr int kGroups = kKpad / 8;
  static constexpr uint32_t kAGroup = kTcM * 16;
  static constexpr uint32_t kBGroup = CIN * 16;
  static constexpr int kBBytes = kKpad * CIN * 2;
  static constexpr int kABytes = kKpad * kTcM * 2;
  static constexpr int kSmem = kBBytes + kABytes;
};
using TcT1 = ConvTcT<32, 3, 32>;
using TcT3 = ConvTcT<32, 2, 2>;
// byte offsets of layers 1..3's transposed images
__host__ __device__ constexpr int tct_img_offset(int li) {
  return (li > 1 ? TcT1::kBBytes : 0) + (li > 2 ? TcT1::kBBytes : 0) + (li > 3 ? TcT3::kBBytes : 0);
}
constexpr int kTcWPos = 64;      // positions per step: four MMAs of K = 16
constexpr int kTcWChunk = 1024;  // positions per CTA
__host__ __device__ constexpr int tc_mtiles(int kw) { return (kw + kTcM - 1) / kTcM; }
int64_t tc_wchunks(int n, const Layer& L) {
  return ((int64_t)n * L.hout * L.hout + kTcWChunk - 1) / kTcWChunk;
}
// Floats of the partial-gradient buffer for n pairs (the largest layer's).
size_t tc_wpart_floats(int n) {
  size_t m = 0;
  const int kw[4] = {18, 288, 288, 128}, nn[4] = {32, 32, 32, 16};
  for (int li = 0; li < 4; ++li)
    m = std::max(m, (size_t)tc_wchunks(n, cnn_layer(li)) * (tc_mtiles(kw[li]) * kTcM + 1) * nn[li]);
  return m;
}


// Workspace layout (byte offsets) for n pairs.
struct CnnWs {
  size_t x0, a1, a2, a3, z4, k, wimg, dz4, dz3, dz2, dz1, grad, lossp, wtimg, wpart, total;
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
    L.wtimg = take(tct_img_offset(4));
    L.wpart = take(tc_wpart_floats(n) * 4);
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
// cells are read once, coalesced (a thread per input column, three channels'
// loads in flight together), weighted by their overlaps and summed over rows
// and channels into a shared column profile (dynamic shared memory, one float
// per input column); each output cell then sums its columns' profile with the
// column overlaps.  Widths up to kCnnMaxW.
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
    int ch = 0;
    for (; ch + 3 <= fr.c; ch += 3) {
      // three channels' loads in flight together; summed in channel order
      const In* row = base + (int64_t)ch * fr.cs + (int64_t)r * fr.rs + threadIdx.x;
      float a[3][kCnnColsPT];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < kCnnColsPT; ++j)
          a[k][j] = ((int)threadIdx.x + j * kCnnThreads < fr.w)
                        ? (float)__ldg(row + k * fr.cs + j * kCnnThreads)
                        : 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < kCnnColsPT; ++j) v[j] += a[k][j];
    }
    for (; ch < fr.c; ++ch) {
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
    if (c < fr.w && CBP_CHECK(c < kCnnMaxW, 6)) prof[c] = col[j];
  }
}

#ifndef CBP_CNN_INPUT_BLOCKS
#define CBP_CNN_INPUT_BLOCKS 4   // resident blocks per SM the register budget is set for
#endif
__global__ void __launch_bounds__(kCnnThreads, CBP_CNN_INPUT_BLOCKS)
k_cnn_input_rows(FrameDesc f1, FrameDesc f2, bf16* x0) {
  extern __shared__ float prof[];   // max(f1.w, f2.w) columns
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
          if (CBP_CHECK(ci0 + 7 < CIN && (int64_t)iy * L.hin + ix < plane, 0))
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
    if (CBP_CHECK(tc::kmajor_offset(kTcM, m, 8 * g) + 16 <= (uint32_t)C::kABytes, 1))
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

__device__ __forceinline__ uint32_t bf16_bits(float v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16(v));
}

// Input gradients on the tensor cores, an implicit GEMM over the layer's
// input positions i (128 per CTA):
//   dx[n][ci][i] = [x[n][ci][i] > 0] sum_k G[i][k] W^T[ci][k],
// k = (u KS + v) COUT + co, G[i][k] = dy[n][co][oy][ox] where iy + p - u = oy s
// and ix + p - v = ox s land on an output position (zero elsewhere: the
// strided transpose of the forward product), rounded to BF16, and
// W^T[ci][k] = w[co][ci][u][v] in BF16 (k_conv_wt_images).  The mask (the
// ReLU of the layer's input) turns it into the previous layer's
// pre-activation gradient.
template <int CIN, int KS, int COUT>
__device__ void conv_wt_image(const float* prm, const Layer& L, uint8_t* img) {
  using C = ConvTcT<CIN, KS, COUT>;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < CIN * C::kKpad; i += gridDim.x * blockDim.x) {
    const int ci = i / C::kKpad, k = i - ci * C::kKpad;
    float w = 0.f;
    if (k < C::kK) {
      const int tap = k / COUT, co = k - tap * COUT;
      w = prm[L.woff + (co * CIN + ci) * KS * KS + tap];
    }
    *(bf16*)(img + tc::kmajor_offset(CIN, ci, k)) = __float2bfloat16(w);
  }
}
__global__ void k_conv_wt_images(const float* prm, uint8_t* img) {
  switch (blockIdx.y) {
    case 0: conv_wt_image<32, 3, 32>(prm, cnn_layer(1), img + tct_img_offset(1)); break;
    case 1: conv_wt_image<32, 3, 32>(prm, cnn_layer(2), img + tct_img_offset(2)); break;
    default: conv_wt_image<32, 2, 2>(prm, cnn_layer(3), img + tct_img_offset(3)); break;
  }
}

template <int CIN, int KS, int COUT>
__global__ void __launch_bounds__(kTcThreads) k_conv_bwd_data_tc(const float* __restrict__ dy,
                                                                  const uint8_t* __restrict__ wtimg,
                                                                  const bf16* __restrict__ xact,
                                                                  float* __restrict__ dx, Layer L, int* err) {
  using C = ConvTcT<CIN, KS, COUT>;
  extern __shared__ __align__(128) uint8_t tsm[];
  __shared__ uint64_t done;
  __shared__ uint32_t tslot;
  uint8_t* sB = tsm;
  uint8_t* sA = tsm + C::kBBytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = blockIdx.y, nin = L.hin * L.hin, hw = L.hout * L.hout, m0 = blockIdx.x * kTcM;

  if (warp == 0) tc::tmem_alloc(&tslot, kTcCols);
  if (tid == 0) tc::bar_init(&done, 1);
  for (int i = tid; i < C::kBBytes / 16; i += kTcThreads)
    ((uint4*)sB)[i] = __ldg((const uint4*)wtimg + i);
  const float* dyn = dy + (int64_t)n * COUT * hw;
#pragma unroll 2
  for (int c = tid; c < kTcM * C::kGroups; c += kTcThreads) {
    const int m = c & (kTcM - 1), g = c / kTcM;
    const int i = m0 + m;
    uint32_t q[4] = {0u, 0u, 0u, 0u};
    if (i < nin) {
      const int iy = i / L.hin, ix = i - iy * L.hin;
      if constexpr (COUT % 8 == 0) {   // the group is 8 channels of one tap
        const int tap = g / (COUT / 8), co0 = (g - tap * (COUT / 8)) * 8;
        const int u = tap / KS, v = tap - u * KS;
        const int ty = iy + L.p - u, tx = ix + L.p - v;
        if (tap < KS * KS && ty >= 0 && tx >= 0 && ty % L.s == 0 && tx % L.s == 0 &&
            ty / L.s < L.hout && tx / L.s < L.hout) {
          const float* pg = dyn + (int64_t)co0 * hw + (ty / L.s) * L.hout + tx / L.s;
          if (CBP_CHECK(co0 + 7 < COUT && (ty / L.s) * L.hout + tx / L.s < hw, 3))
#pragma unroll
            for (int e = 0; e < 8; ++e) q[e >> 1] |= bf16_bits(__ldg(pg + e * hw)) << (16 * (e & 1));
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = g * 8 + e;
          const int tap = k / COUT, co = k - tap * COUT;
          const int u = tap / KS, v = tap - u * KS;
          const int ty = iy + L.p - u, tx = ix + L.p - v;
          if (tap < KS * KS && ty >= 0 && tx >= 0 && ty % L.s == 0 && tx % L.s == 0 &&
              ty / L.s < L.hout && tx / L.s < L.hout)
            q[e >> 1] |= bf16_bits(__ldg(dyn + (int64_t)co * hw + (ty / L.s) * L.hout + tx / L.s))
                         << (16 * (e & 1));
        }
      }
    }
    if (CBP_CHECK(tc::kmajor_offset(kTcM, m, 8 * g) + 16 <= (uint32_t)C::kABytes, 2))
      *(uint4*)(sA + tc::kmajor_offset(kTcM, m, 8 * g)) = make_uint4(q[0], q[1], q[2], q[3]);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    const uint32_t a0 = tc::saddr(sA), b0 = tc::saddr(sB);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, CIN);
#pragma unroll 1
    for (int s = 0; s < C::kKpad / 16; ++s)
      tc::mma_bf16(tmem, tc::sdesc(a0 + 2 * s * C::kAGroup, C::kAGroup, 128),
                   tc::sdesc(b0 + 2 * s * C::kBGroup, C::kBGroup, 128), idesc, s > 0);
    tc::mma_commit(&done);
  }
  const bool arrived = tc::bar_wait(&done, 0, kTcWaitLimit);
  const bool late = __syncthreads_or(!arrived);
  if (late) {
    if (tid == 0 && err) atomicOr(err, 1);
    if (!arrived) tc::bar_wait(&done, 0, kTcWaitLimit);
  }
  tc::fence_after_sync();
  const int quarter = warp & 3, half = warp >> 2;
  float v[16];
  if (!late) {
    tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + half * 16, v);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __int_as_float(0x7fc00000);
  }
  const int i = m0 + quarter * 32 + lane;
  if (i < nin) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int64_t at = ((int64_t)n * CIN + half * 16 + j) * nin + i;
      dx[at] = __bfloat162float(xact[at]) > 0.f ? v[j] : 0.f;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, kTcCols);
  }
  static_assert(CIN == 32, "one output channel per accumulator column, 16 per warp half");
}

// Weight gradients on the tensor cores, an implicit GEMM whose reduction runs
// over the output positions o of all pairs:
//   D[k][co] = sum_o X[k][o] dY[co][o],
// k = (u KS + v) CIN + ci a weight's tap and input channel, X[k][o] = the layer
// input x[n][ci][oy s - p + u][ox s - p + v] (zero outside), dY = dy rounded to
// BF16.  A CTA takes 128 rows of k (M) and kTcWChunk positions, in steps of
// kTcWPos positions through two shared-memory buffers: the MMAs of one step run
// while the other buffer is filled, each buffer's MMAs completing on its own
// mbarrier before it is refilled.  The bias gradients sum dy itself in FP32
// (the CTAs of the first row tile, from the values they stage).  Each CTA
// writes its partials; a second kernel sums them over the position chunks in
// a fixed order (deterministic) into the gradient vector.
template <int CIN, int KS, int N>
__global__ void __launch_bounds__(kTcThreads) k_conv_bwd_w_tc(const float* __restrict__ dy,
                                                               const bf16* __restrict__ x,
                                                               float* __restrict__ part, Layer L,
                                                               int npairs, int* err) {
  constexpr int KW = KS * KS * CIN;
  constexpr int kABytes = kTcM * kTcWPos * 2, kBBytes = N * kTcWPos * 2;
  extern __shared__ __align__(128) uint8_t tsm[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int hw = L.hout * L.hout;
  const int64_t P = (int64_t)npairs * hw;
  const int kk0 = blockIdx.x * kTcM;
  const int64_t pbeg = (int64_t)blockIdx.y * kTcWChunk, pend = min(P, pbeg + kTcWChunk);
  const int steps = (int)((pend - pbeg + kTcWPos - 1) / kTcWPos);
  const unsigned short* xs = reinterpret_cast<const unsigned short*>(x);

  __shared__ float bred[8][N];
  float bsum = 0.f;   // this thread's FP32 share of the bias gradient
  if (warp == 0) tc::tmem_alloc(&tslot, kTcCols);
  if (tid == 0) {
    tc::bar_init(&bars[0], 1);
    tc::bar_init(&bars[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(kTcM, N);
  bool ok = true, late = false;
  int issued = 0;
#pragma unroll 1
  for (int t = 0; t < steps; ++t) {
    const int b = t & 1;
    uint8_t* sA = tsm + b * (kABytes + kBBytes);
    uint8_t* sB = sA + kABytes;
    // the MMAs of step t - 2 read this buffer
    if (t >= 2) ok = tc::bar_wait(&bars[b], ((t - 2) >> 1) & 1, kTcWaitLimit) && ok;
    const int64_t ob = pbeg + (int64_t)t * kTcWPos;
    // X rows kk0 + r, positions ob + 8 g + e; a warp's lanes are 32 consecutive rows
    for (int c = tid; c < kTcM * (kTcWPos / 8); c += kTcThreads) {
      const int r = c & (kTcM - 1), g = c / kTcM, kk = kk0 + r;
      uint32_t q[4] = {0u, 0u, 0u, 0u};
      if (kk < KW) {
        const int tap = kk / CIN, ci = kk - tap * CIN;
        const int u = tap / KS, v = tap - u * KS;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int64_t o = ob + 8 * g + e;
          if (o >= pend) break;
          const int pr = (int)(o / hw), loc = (int)(o - (int64_t)pr * hw);
          const int oy = loc / L.hout, ox = loc - oy * L.hout;
          const int iy = oy * L.s - L.p + u, ix = ox * L.s - L.p + v;
          if (iy >= 0 && iy < L.hin && ix >= 0 && ix < L.hin)
            q[e >> 1] |= (uint32_t)__ldg(xs + (((int64_t)pr * CIN + ci) * L.hin + iy) * L.hin + ix)
                         << (16 * (e & 1));
        }
      }
      if (CBP_CHECK(tc::kmajor_offset(kTcM, r, 8 * g) + 16 <= (uint32_t)kABytes, 4))
        *(uint4*)(sA + tc::kmajor_offset(kTcM, r, 8 * g)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
    // dY rows co, the same positions
    for (int c = tid; c < N * (kTcWPos / 8); c += kTcThreads) {
      const int co = c % N, g = c / N;
      uint32_t q[4] = {0u, 0u, 0u, 0u};
      if (co < L.cout) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int64_t o = ob + 8 * g + e;
          if (o >= pend) break;
          const int pr = (int)(o / hw), loc = (int)(o - (int64_t)pr * hw);
          const float d = __ldg(dy + ((int64_t)pr * L.cout + co) * hw + loc);
          bsum += d;
          q[e >> 1] |= bf16_bits(d) << (16 * (e & 1));
        }
      }
      if (CBP_CHECK(tc::kmajor_offset(N, co, 8 * g) + 16 <= (uint32_t)kBBytes, 5))
        *(uint4*)(sB + tc::kmajor_offset(N, co, 8 * g)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    late = __syncthreads_or(!ok);
    tc::fence_after_sync();
    if (late) break;
    if (tid == 0) {
      const uint32_t a0 = tc::saddr(sA), b0 = tc::saddr(sB);
#pragma unroll
      for (int s = 0; s < kTcWPos / 16; ++s)
        tc::mma_bf16(tmem, tc::sdesc(a0 + 2 * s * kTcM * 16, kTcM * 16, 128),
                     tc::sdesc(b0 + 2 * s * N * 16, N * 16, 128), idesc, t > 0 || s > 0);
      tc::mma_commit(&bars[b]);
    }
    ++issued;
  }
  // the bias partial of this chunk: the eight position groups in order
  // (every thread c < 8 N staged one (co, g) in each step)
  if (tid < 8 * N) bred[tid / N][tid % N] = bsum;
  __syncthreads();
  if (blockIdx.x == 0 && tid < N) {
    float b = 0.f;
#pragma unroll
    for (int g = 0; g < 8; ++g) b += bred[g][tid];
    part[(int64_t)gridDim.y * gridDim.x * kTcM * N + (int64_t)blockIdx.y * N + tid] = b;
  }
  // the last commit completes after every MMA issued before it
  bool fin = true;
  if (issued > 0) fin = tc::bar_wait(&bars[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kTcWaitLimit);
  const bool bad = __syncthreads_or(!fin) || late;
  if (bad) {
    // report, wait once more (bounded) for the MMAs in flight, leave NaN partials
    if (tid == 0 && err) atomicOr(err, 1);
    if (issued > 0 && !fin)
      tc::bar_wait(&bars[(issued - 1) & 1], ((issued - 1) >> 1) & 1, kTcWaitLimit);
  }
  tc::fence_after_sync();
  const int quarter = warp & 3, half = warp >> 2;
  if (half * 16 < N) {
    float v[16];
    if (!bad) {
      tc::tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + half * 16, v);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = __int_as_float(0x7fc00000);
    }
    float4* o = (float4*)(part + (((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * kTcM + quarter * 32 +
                                  lane) * N + half * 16);
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_free(tmem, kTcCols);
  }
}

// The gradient vector from the partials, summed over the position chunks in
// order: weights [co][ci][u][v] from rows k < KS^2 CIN, then the biases.
template <int CIN, int KS, int N>
__global__ void k_conv_bwd_w_sum(const float* __restrict__ part, float* __restrict__ grad, Layer L,
                                 int nchunks, int mtiles) {
  constexpr int KW = KS * KS * CIN;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (KW + 1) * L.cout) return;
  const int kk = idx / L.cout, co = idx - kk * L.cout;
  float s = 0.f;
  if (kk < KW) {
    for (int c = 0; c < nchunks; ++c)
      s += part[(((int64_t)c * mtiles + kk / kTcM) * kTcM + kk % kTcM) * N + co];
  } else {
    const float* bp = part + (int64_t)nchunks * mtiles * kTcM * N;
    for (int c = 0; c < nchunks; ++c) s += bp[(int64_t)c * N + co];
  }
  if (kk < KW) {
    const int tap = kk / CIN, ci = kk - tap * CIN;
    grad[L.woff + (co * CIN + ci) * KS * KS + tap] = s;
  } else {
    grad[L.boff + co] = s;
  }
}

template <int CIN, int KS, int N>
void run_bwd_w_tc(const float* dy, const bf16* x, float* part, float* grad, int li, int n, int* err,
                  cudaStream_t st) {
  const Layer L = cnn_layer(li);
  constexpr int KW = KS * KS * CIN;
  const int mt = tc_mtiles(KW);
  const int nch = (int)tc_wchunks(n, L);
  const int sm = 2 * (kTcM * kTcWPos * 2 + N * kTcWPos * 2);
  auto kfn = k_conv_bwd_w_tc<CIN, KS, N>;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  kfn<<<dim3(mt, nch), kTcThreads, sm, st>>>(dy, x, part, L, n, err);
  k_conv_bwd_w_sum<CIN, KS, N><<<((KW + 1) * L.cout + 255) / 256, 256, 0, st>>>(part, grad, L, nch, mt);
}

template <int CIN, int KS, int COUT>
void run_bwd_data_tc(const float* dy, const uint8_t* wt, const bf16* xact, float* dx, int li, int n,
                     int* err, cudaStream_t st) {
  using C = ConvTcT<CIN, KS, COUT>;
  const Layer L = cnn_layer(li);
  auto kfn = k_conv_bwd_data_tc<CIN, KS, COUT>;
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem);
  kfn<<<dim3((L.hin * L.hin + kTcM - 1) / kTcM, n), kTcThreads, C::kSmem, st>>>(
      dy, wt + tct_img_offset(li), xact, dx, L, err);
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
    k_cnn_input_rows<<<dim3(kCnnSide, 2, n), kCnnThreads, sizeof(float) * std::max(b1.w, b2.w), st>>>(
        b1, b2, x0);
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
  uint8_t* wt = (uint8_t*)(ws + L.wtimg);
  float* part = (float*)(ws + L.wpart);
  k_conv_wt_images<<<dim3(8, 3), 256, 0, st>>>(prm, wt);
  // layer by layer from the head: weight gradients, then the input gradient
  run_bwd_w_tc<32, 2, 16>(dz[3], a[2], part, grad, 3, n, nullptr, st);
  run_bwd_data_tc<32, 2, 2>(dz[3], wt, a[2], dz[2], 3, n, nullptr, st);
  run_bwd_w_tc<32, 3, 32>(dz[2], a[1], part, grad, 2, n, nullptr, st);
  run_bwd_data_tc<32, 3, 32>(dz[2], wt, a[1], dz[1], 2, n, nullptr, st);
  run_bwd_w_tc<32, 3, 32>(dz[1], a[0], part, grad, 1, n, nullptr, st);
  run_bwd_data_tc<32, 3, 32>(dz[1], wt, a[0], dz[0], 1, n, nullptr, st);
  run_bwd_w_tc<2, 3, 32>(dz[0], x0, part, grad, 0, n, nullptr, st);
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
  cbp::NvtxScope range("cbp_cnn_forward");
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
  cbp::NvtxScope range("cbp_cnn_train_step");
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
