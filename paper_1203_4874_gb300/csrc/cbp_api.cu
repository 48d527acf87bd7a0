// C ABI of libcbp (declared in include/cbp.h): contexts, workspaces and the
// batched estimation / deblurring entry points.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>
#include "cbp.h"
#include "cbp_common.cuh"
#include "cbp_internal.h"
#if defined(CBP_DEBUG_ERRORS) || defined(CBP_TIMELINE)
#include <cstdio>
#endif
#include "cbp_serve.h"
#include "cbp_nvtx.h"

namespace cbp {

// Device memory accounting of a context (workspaces and serving slots).
bool Ctx::reserve(size_t bytes) {
  std::lock_guard<std::mutex> g(mem_mu);
  if (used + bytes > budget) return false;
  used += bytes;
  return true;
}
void Ctx::release(size_t bytes) {
  std::lock_guard<std::mutex> g(mem_mu);
  used -= std::min(used, bytes);
}

cudaEvent_t Prof::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
void Prof::begin(int, cudaStream_t st, cudaEvent_t* a) {
  *a = get();
  cudaEventRecord(*a, st);
}
void Prof::end(int stage, cudaStream_t st, cudaEvent_t a, int nkernels) {
  cudaEvent_t b = get();
  cudaEventRecord(b, st);
  recs.push_back({stage, a, b});
  launches[stage] += nkernels;
}

// Grow the synchronous-API workspace to `bytes` (stream-ordered on `st`).
cbp_status Ctx::ensure_ws(size_t bytes, cudaStream_t st) {
  if (bytes <= ws_size) return CBP_OK;
  if (!reserve(bytes)) return CBP_ERR_BUDGET;
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    release(bytes);
    return CBP_ERR_OOM;
  }
  if (ws) {
    cudaFreeAsync(ws, st);
    release(ws_size);
  }
  ws = (char*)p;
  ws_size = bytes;
  ++ws_gen;
  return CBP_OK;
}

cbp_status Ctx::ensure_chunk_streams() {
  if (chunk_ready) return CBP_OK;
  for (int i = 0; i < kChunkStreams; ++i)
    if (cudaStreamCreateWithFlags(&chunk_st[i], cudaStreamNonBlocking) != cudaSuccess)
      return CBP_ERR_CUDA;
  if (cudaStreamCreateWithFlags(&io_st, cudaStreamNonBlocking) != cudaSuccess) return CBP_ERR_CUDA;
  int prio_lo = 0, prio_hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) return CBP_ERR_CUDA;
  for (int i = 0; i < kChunkStreams; ++i)
    if (cudaStreamCreateWithPriority(&solve_st[i], cudaStreamNonBlocking, prio_hi) != cudaSuccess)
      return CBP_ERR_CUDA;
  for (int i = 0; i < kMaxChunks; ++i)
    if (cudaEventCreateWithFlags(&fork_ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join_ev[i], cudaEventDisableTiming) != cudaSuccess)
      return CBP_ERR_CUDA;
  for (int i = 0; i <= kMaxChunks; ++i)
    if (cudaEventCreateWithFlags(&chunk_ev[i], cudaEventDisableTiming) != cudaSuccess)
      return CBP_ERR_CUDA;
  for (int i = 0; i < kMaxChunks; ++i)
    if (cudaEventCreateWithFlags(&io_ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&read_ev[i], cudaEventDisableTiming) != cudaSuccess)
      return CBP_ERR_CUDA;
  chunk_ready = true;
  return CBP_OK;
}

// Grow the standalone network calls' workspace (stream-ordered on `st`).
cbp_status Ctx::ensure_cnn_ws(size_t bytes, cudaStream_t st) {
  if (bytes <= cnn_ws_size) return CBP_OK;
  if (!reserve(bytes)) return CBP_ERR_BUDGET;
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    release(bytes);
    return CBP_ERR_OOM;
  }
  if (cnn_ws) {
    cudaFreeAsync(cnn_ws, st);
    release(cnn_ws_size);
  }
  cnn_ws = (char*)p;
  cnn_ws_size = bytes;
  return CBP_OK;
}

// Check-word readers of the source files (bounds-checked builds).
namespace {
unsigned (*&check_reader(int id))(bool) {
  static unsigned (*readers[kChkWords])(bool) = {};
  return readers[id];
}
}  // namespace
void register_check_word(int id, unsigned (*read)(bool)) {
  if (id >= 0 && id < kChkWords) check_reader(id) = read;
}

// Range names of the stages (cbp_stage order).
const char* stage_label(int stage) {
  static const char* const names[CBP_NUM_STAGES] = {
      "cbp.eval",     "cbp.sample_solve", "cbp.scale_solve", "cbp.kernel_spectra",
      "cbp.row_fft",  "cbp.col_deconv",   "cbp.row_ifft",    "cbp.h2d",
      "cbp.d2h",      "cbp.proposal",     "cbp.gate"};
  return stage >= 0 && stage < CBP_NUM_STAGES ? names[stage] : "cbp.stage";
}

// Enqueue the whole path of one plan on `st` with workspace `wsp`.
cbp_status run_plan(const Plan& p, const cbp_frames* b1, const cbp_frames* b2,
                    const cbp_params* prm, void* k1, void* k2, void* latent, bool deblur,
                    char* wsp, cudaStream_t st, Prof* prof, const PtrTables* tabs,
                    const float* cnn_w, bool h2d_done, cudaEvent_t after_read,
                    cudaStream_t solve, cudaEvent_t fork, cudaEvent_t join, bool tw_ready) {
  cudaEvent_t ev = nullptr;
  cudaStream_t cur = st;   // the stream stages are timed on
  // an NVTX range per stage; one still open at an error return is closed here
  struct OpenRanges {
    int n = 0;
    ~OpenRanges() {
      for (; n > 0; --n) nvtx_pop();
    }
  } ranges;
  auto begin = [&](int stage) {
    nvtx_push(stage_label(stage));
    ++ranges.n;
    if (prof) prof->begin(stage, cur, &ev);
  };
  auto end = [&](int stage, int nk) {
    if (prof) prof->end(stage, cur, ev, nk);
    nvtx_pop();
    --ranges.n;
  };
  const bool host_io = prm->flags & CBP_FLAG_HOST_IO;
  const bool kin = deblur && (prm->flags & CBP_FLAG_KERNELS_IN);
  const int f64 = b1->dtype == CBP_F64;
  const int kf64 = f64 || (prm->flags & CBP_FLAG_KERNELS_F64);
  const size_t es = f64 ? 8 : 4;
  const size_t kes = kf64 ? 8 : 4;
  FrameDesc d1, d2;
  void* k1d = k1;
  void* k2d = k2;
  void* latd = latent;
  if (host_io) {
    begin(CBP_STAGE_H2D);
    const cbp_frames* bs[2] = {b1, b2};
    for (int k = 0; k < 2; ++k) {
      const cbp_frames* b = bs[k];
      const int64_t rs = b->row_stride ? b->row_stride : b->w;
      const int64_t cs = b->chan_stride ? b->chan_stride : (int64_t)b->h * rs;
      const int64_t fs = b->frame_stride ? b->frame_stride : (int64_t)b->c * cs;
      if (rs != b->w || cs != (int64_t)b->h * b->w || fs != (int64_t)b->c * cs)
        return CBP_ERR_INVALID_ARG;  // host I/O takes contiguous batches
      const size_t bytes = (size_t)b->n * b->c * b->h * b->w * es;
      if (!h2d_done &&
          cudaMemcpyAsync(wsp + p.off_io_b[k], b->data, bytes, cudaMemcpyHostToDevice, st) !=
              cudaSuccess)
        return CBP_ERR_CUDA;
    }
    d1 = frame_desc(b1, wsp + p.off_io_b[0]);
    d2 = frame_desc(b2, wsp + p.off_io_b[1]);
    k1d = k1 ? wsp + p.off_io_k[0] : nullptr;
    k2d = k2 ? wsp + p.off_io_k[1] : nullptr;
    latd = wsp + p.off_io_lat;
    if (kin && !h2d_done) {
      if (cudaMemcpyAsync(k1d, k1, (size_t)p.n * p.t1 * p.t1 * kes, cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(k2d, k2, (size_t)p.n * p.t2 * p.t2 * kes, cudaMemcpyHostToDevice, st) !=
              cudaSuccess)
        return CBP_ERR_CUDA;
    }
    end(CBP_STAGE_H2D, 0);
  } else {
    d1 = frame_desc(b1, nullptr);
    d2 = frame_desc(b2, nullptr);
    if (tabs) {
      d1.tab = tabs->b1;
      d2.tab = tabs->b2;
    }
  }
  cudaMemsetAsync(wsp + p.off_bad, 0, (size_t)p.n * sizeof(int), st);
  cudaMemsetAsync(wsp + p.off_err, 0, sizeof(int), st);
  if (kin) {
    if ((!k1d || !k2d) && !(tabs && tabs->k1 && tabs->k2)) return CBP_ERR_INVALID_ARG;
    begin(CBP_STAGE_SCALE_SOLVE);
    launch_kernels_in(p, wsp, k1d, k2d, kf64, st, tabs ? tabs->k1 : nullptr,
                      tabs ? tabs->k2 : nullptr);
    end(CBP_STAGE_SCALE_SOLVE, 1);
  }
  if (p.learned && !cnn_w) return CBP_ERR_INVALID_ARG;   // no weights loaded
  const bool fft = deblur || p.learned;
  if (p.learned) {
    // learned path: the network's proposal, written where the estimate goes
    begin(CBP_STAGE_PROPOSAL);
    cnn_forward(d1, d2, p.n, cnn_w, wsp + p.off_cnn, st, nullptr, (int*)(wsp + p.off_err));
    cnn_to_kd(wsp + p.off_cnn, p.n, (double*)(wsp + p.off_kd), st);
    end(CBP_STAGE_PROPOSAL, 8);
  }
  if (fft) {
    if (!tw_ready) {
      begin(CBP_STAGE_KERNEL_SPECTRA);   // FFT twiddle tables
      init_twiddles(p, wsp, st);
      end(CBP_STAGE_KERNEL_SPECTRA, 4);
    }
    // one read of the frames: A1 folds and the A6 forward row FFTs together
    begin(CBP_STAGE_ROW_FFT);
    launch_row_pass(p, d1, d2, wsp, st, !kin, true);
    end(CBP_STAGE_ROW_FFT, 1);
  }
  if (after_read && cudaEventRecord(after_read, st) != cudaSuccess) return CBP_ERR_CUDA;
  if (p.learned) {
    // consistency residual of the proposal; accepted pairs skip the solves
    begin(CBP_STAGE_GATE);
    if (p.col_fused) {
      // the proposal's deconvolution with the residual sums (its spectrum stands
      // for accepted pairs; the column pass below redoes the rejected ones)
      launch_col_gate_fused(p, wsp, st);
    } else {
      launch_kernel_spectra(p, wsp, st);
      launch_residual_gate(p, wsp, st);
    }
    end(CBP_STAGE_GATE, 3);
  }
  if (!kin) {
    // the latency-bound estimation, on the high-priority stream when given
    const bool forked = solve && fork && join;
    if (forked && (cudaEventRecord(fork, st) != cudaSuccess ||
                   cudaStreamWaitEvent(solve, fork, 0) != cudaSuccess))
      return CBP_ERR_CUDA;
    cudaStream_t es = forked ? solve : st;
    cur = es;
    begin(CBP_STAGE_EVAL);
    if (fft) launch_fold_dft(p, wsp, es);
    else launch_eval(p, d1, d2, wsp, es);
    end(CBP_STAGE_EVAL, fft ? 1 : 2);
    begin(CBP_STAGE_SAMPLE_SOLVE);
    launch_sample_solve(p, wsp, es);
    end(CBP_STAGE_SAMPLE_SOLVE, 1);
    begin(CBP_STAGE_SCALE_SOLVE);
    launch_scale_solve(p, wsp, k1d, k2d, kf64, es, tabs ? tabs->k1 : nullptr,
                       tabs ? tabs->k2 : nullptr);
    end(CBP_STAGE_SCALE_SOLVE, 1);
    cur = st;
    if (forked && (cudaEventRecord(join, solve) != cudaSuccess ||
                   cudaStreamWaitEvent(st, join, 0) != cudaSuccess))
      return CBP_ERR_CUDA;
  }
  if (deblur) {
    if (!p.col_fused) {
      begin(CBP_STAGE_KERNEL_SPECTRA);
      launch_kernel_spectra(p, wsp, st);
      end(CBP_STAGE_KERNEL_SPECTRA, 1);
    }
    begin(CBP_STAGE_COL_DECONV);
    launch_col_deconv(p, wsp, st);
    end(CBP_STAGE_COL_DECONV, p.col_fused ? 2 : 1);   // fused: the kernels' row transforms first
    begin(CBP_STAGE_ROW_IFFT);
    launch_row_ifft(p, wsp, latd, f64, st, tabs ? tabs->lat : nullptr);
    end(CBP_STAGE_ROW_IFFT, 1);
  }
  if (host_io) {
    begin(CBP_STAGE_D2H);
    if (deblur &&
        cudaMemcpyAsync(latent, latd, (size_t)p.n * p.C * p.H * p.W * es, cudaMemcpyDeviceToHost,
                        st) != cudaSuccess)
      return CBP_ERR_CUDA;
    if (!kin && k1 &&
        cudaMemcpyAsync(k1, k1d, (size_t)p.n * p.t1 * p.t1 * kes, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
      return CBP_ERR_CUDA;
    if (!kin && k2 &&
        cudaMemcpyAsync(k2, k2d, (size_t)p.n * p.t2 * p.t2 * kes, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
      return CBP_ERR_CUDA;
    end(CBP_STAGE_D2H, 0);
  }
  const cudaError_t ce = cudaGetLastError();
#ifdef CBP_DEBUG_ERRORS
  if (ce != cudaSuccess) fprintf(stderr, "cbp: %s\n", cudaGetErrorString(ce));
#endif
  if (ce != cudaSuccess) return CBP_ERR_CUDA;
  return CBP_OK;
}

}  // namespace cbp

using cbp::Ctx;
using cbp::Plan;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

cbp_status copy_stages(const Plan& p, const char* ws, const cbp_stage_out* o, cudaStream_t st) {
  if (!o) return CBP_OK;
  const size_t te = 16;   // double samples on both paths
  const size_t n = p.n, C = p.C, ns = p.ns;
  struct Item { void* dst; size_t off, bytes; };
  const Item items[] = {
      {o->p_z2[0], p.off_pz2[0], n * C * ns * p.H1 * te},
      {o->p_z2[1], p.off_pz2[1], n * C * ns * p.H2 * te},
      {o->p_z1[0], p.off_pz1[0], n * C * ns * p.W1 * te},
      {o->p_z1[1], p.off_pz1[1], n * C * ns * p.W2 * te},
      {o->sample_diag, p.off_sdiag, n * 2 * ns * 4 * 8},
      {o->lifted, p.off_resid, n * 4 * (size_t)p.M * p.M * 16},
      {o->kernels, p.off_kd, n * (size_t)(p.t1 * p.t1 + p.t2 * p.t2) * 8},
  };
  for (const Item& it : items)
    if (it.dst && cudaMemcpyAsync(it.dst, ws + it.off, it.bytes, cudaMemcpyDeviceToDevice, st) !=
                      cudaSuccess)
      return CBP_ERR_CUDA;
  // null vectors: workspace layout [n][2][ns][nn] -> two [n][ns][nn] arrays
  void* xs[2] = {o->x_z2, o->x_z1};
  for (int ps = 0; ps < 2; ++ps)
    if (xs[ps] && cudaMemcpy2DAsync(xs[ps], ns * p.nn * 16, ws + p.off_x + ps * ns * p.nn * 16,
                                    2 * ns * p.nn * 16, ns * p.nn * 16, n,
                                    cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return CBP_ERR_CUDA;
  return CBP_OK;
}

// A batch is split into up to kChunks chunks (kIoChunks with host I/O) of
// about n / chunks pairs, at least kMinChunkPairs (host I/O: the last three
// smaller)
// (each with its own plan and workspace region) on the context's internal
// streams: the chunks' kernels fill each other's idle
// SMs and tails (the scale solve, for one, runs one block per pair).  Pairs
// are independent, so the results do not depend on the split.
#ifndef CBP_CHUNKS
#define CBP_CHUNKS 2     // chunks of a device-resident call (measured with the current kernels: 2: 6.58, 3: 6.64, 4: 6.73 ms per 60-pair step)
#endif
constexpr int kChunks = CBP_CHUNKS;
constexpr int kIoChunks = Ctx::kMaxChunks;
constexpr int kMinChunkPairs = 8;

// Host I/O takes contiguous batches.
bool contiguous(const cbp_frames* b) {
  const int64_t rs = b->row_stride ? b->row_stride : b->w;
  const int64_t cs = b->chan_stride ? b->chan_stride : (int64_t)b->h * rs;
  const int64_t fs = b->frame_stride ? b->frame_stride : (int64_t)b->c * cs;
  return rs == b->w && cs == (int64_t)b->h * b->w && fs == (int64_t)b->c * cs;
}

// The frames / outputs of pairs [start, start + count) of a batch.
cbp_frames frames_slice(const cbp_frames* f, int start, int count) {
  cbp_frames s = *f;
  const int64_t rs = f->row_stride ? f->row_stride : f->w;
  const int64_t cs = f->chan_stride ? f->chan_stride : (int64_t)f->h * rs;
  const int64_t fs = f->frame_stride ? f->frame_stride : (int64_t)f->c * cs;
  const size_t es = f->dtype == CBP_F64 ? 8 : 4;
  s.data = (const char*)f->data + (size_t)start * (size_t)fs * es;
  s.n = count;
  s.row_stride = rs;
  s.chan_stride = cs;
  s.frame_stride = fs;
  return s;
}

// Kernel-size scan of a batch on the device, results copied to the host.
cbp_status size_scan(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                     const cbp_size_params* sprm, int32_t* t1_out, int32_t* t2_out,
                     int32_t* found, double* ratios, int32_t* ncand_out, void* stream) {
  if (!ctx || !t1_out || !t2_out) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cbp::SizePlan sp;
  cbp_status s = cbp::make_size_plan(b1, b2, sprm, &sp);
  if (s != CBP_OK) return s;
  if (ncand_out) *ncand_out = sp.ncand;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(c->api_mu);
  c->tw_key = 0;   // the workspace is laid out differently
  s = c->ensure_ws(sp.total, st);
  if (s != CBP_OK) return s;
  const cbp::FrameDesc d1 = cbp::frame_desc(b1, nullptr), d2 = cbp::frame_desc(b2, nullptr);
  cbp::launch_size_scan(sp, d1, d2, c->ws, st);
  if (cudaGetLastError() != cudaSuccess) return CBP_ERR_CUDA;
  // t out as [n][3] ints on the device: t1, t2, found
  const int* tdev = (const int*)(c->ws + sp.off_t);
  for (int k = 0; k < 3; ++k) {
    int32_t* dst = k == 0 ? t1_out : k == 1 ? t2_out : found;
    if (dst && cudaMemcpy2DAsync(dst, sizeof(int32_t), tdev + k, 3 * sizeof(int), sizeof(int32_t),
                                 sp.n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return CBP_ERR_CUDA;
  }
  if (ratios && cudaMemcpyAsync(ratios, c->ws + sp.off_rmax, (size_t)sp.n * sp.ncand * sizeof(double),
                                cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CBP_ERR_CUDA;
  return CBP_OK;
}

// Draw coprime kernel pairs (kinds ka, kb) for every frame of a batch on the
// device, redrawing in rounds; attempts (device int[n]) ends with the accepted
// draw or -1.
cbp_status draw_coprime_pairs(int n, int ta, int tb, int kind_a, int kind_b, int M, double tol,
                              int max_attempts, int frame0, uint64_t seed, double* ka, double* kb,
                              char* ws, cudaStream_t st) {
  int* active = (int*)ws;
  int* attempt = active + n;
  int* any = attempt + n;
  int* pass = any + 4;
  std::vector<int> ones((size_t)n, 1);
  if (cudaMemcpyAsync(active, ones.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(attempt, 0, (size_t)n * sizeof(int), st) != cudaSuccess)
    return CBP_ERR_CUDA;
  for (int r = 0; r < max_attempts; ++r) {
    cbp::launch_draw_kernels(n, ta, kind_a, frame0, seed, active, attempt, ka, st);
    cbp::launch_draw_kernels(n, tb, kind_b, frame0, seed, active, attempt, kb, st);
    int h_any = 0;
    if (cudaMemsetAsync(any, 0, sizeof(int), st) != cudaSuccess) return CBP_ERR_CUDA;
    cbp::launch_coprime_round(ka, kb, n, ta, tb, M, tol, max_attempts, active, attempt, pass, any, st);
    if (cudaMemcpyAsync(&h_any, any, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CBP_ERR_CUDA;
    if (!h_any) break;
  }
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

cbp_status encrypt_frames(cbp_ctx* ctx, const void* latent, int32_t n, int32_t c, int32_t h,
                          int32_t w, cbp_dtype dtype, const cbp_encrypt_params* prm, double* k1,
                          double* k2, void* b1, void* b2, double* k3, double* k4, void* c1, void* c2,
                          int32_t* attempts, void* stream) {
  if (!ctx || !latent || !prm || !k1 || !k2 || !b1 || !b2 || n < 1 || c < 1 || h < 1 || w < 1 ||
      (dtype != CBP_F32 && dtype != CBP_F64) || !(prm->sigma >= 0.0))
    return CBP_ERR_INVALID_ARG;
  const bool cascade = prm->t3 > 0 || prm->t4 > 0;
  const int ts[4] = {prm->t1, prm->t2, prm->t3, prm->t4};
  for (int i = 0; i < (cascade ? 4 : 2); ++i)
    if (ts[i] < 1 || ts[i] > 32) return CBP_ERR_INVALID_ARG;
  if (cascade && (!k3 || !k4 || !c1 || !c2)) return CBP_ERR_INVALID_ARG;
  const int M1 = prm->m ? prm->m : std::max(prm->t1, prm->t2);
  const int M2 = prm->m ? prm->m : std::max(prm->t3, prm->t4);
  if (M1 < 1 || M1 > cbp::kMaxM || (cascade && (M2 < 1 || M2 > cbp::kMaxM))) return CBP_ERR_INVALID_ARG;
  const int maxa = prm->max_attempts > 0 ? prm->max_attempts : 8;
  const double tol = prm->tol > 0.0 ? prm->tol : 1e-7;
  if (!std::isfinite(tol) || maxa > 255) return CBP_ERR_INVALID_ARG;
  Ctx* cx = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(cx->device);
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(cx->api_mu);
  const int Mmax = std::max(M1, cascade ? M2 : 1);
  const size_t per = (size_t)(2 * n + 4 + n * 2 * (Mmax / 2 + 1)) * sizeof(int);
  cx->tw_key = 0;   // the workspace is laid out differently
  cbp_status s = cx->ensure_ws(2 * ((per + 255) & ~size_t(255)), st);
  if (s != CBP_OK) return s;
  char* wa = cx->ws;
  char* wb = cx->ws + ((per + 255) & ~size_t(255));
  s = draw_coprime_pairs(n, prm->t1, prm->t2, 0, 1, M1, tol, maxa, prm->frame0, prm->seed, k1, k2, wa, st);
  if (s != CBP_OK) return s;
  if (cascade) {
    s = draw_coprime_pairs(n, prm->t3, prm->t4, 2, 3, M2, tol, maxa, prm->frame0, prm->seed, k3, k4, wb,
                           st);
    if (s != CBP_OK) return s;
  }
  // noise keys per batch and stream
  const uint64_t nkey = prm->seed + 0x100000000ull * (uint64_t)(prm->frame0 + 1);
  const int f64 = dtype == CBP_F64;
  cbp::launch_forward_blur(latent, n, c, h, w, f64, k1, prm->t1, prm->sigma, nkey + 1, b1, st);
  cbp::launch_forward_blur(latent, n, c, h, w, f64, k2, prm->t2, prm->sigma, nkey + 2, b2, st);
  if (cascade) {
    const int hb = h + prm->t1 - 1, wb1 = w + prm->t1 - 1;
    cbp::launch_forward_blur(b1, n, c, hb, wb1, f64, k3, prm->t3, 0.0, 0, c1, st);
    cbp::launch_forward_blur(b1, n, c, hb, wb1, f64, k4, prm->t4, 0.0, 0, c2, st);
  }
  if (attempts) {
    if (cudaMemcpyAsync(attempts, (int*)wa + n, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        (cascade && cudaMemcpyAsync(attempts + n, (int*)wb + n, (size_t)n * sizeof(int),
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess))
      return CBP_ERR_CUDA;
  }
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

cbp_status call_path(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                     const cbp_params* prm, void* k1, void* k2, void* latent, cbp_diag* diag,
                     void* stream, bool deblur, const cbp_stage_out* stages = nullptr) {
  if (!ctx) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  Plan p;
  cbp_status s = cbp::make_plan(b1, b2, prm, &p);
  if (s != CBP_OK) return s;
  p.pz_all = stages ? 1 : 0;   // the stage outputs hold double samples
  if (deblur && !latent) return CBP_ERR_INVALID_ARG;
  if (!deblur && (!k1 || !k2)) return CBP_ERR_INVALID_ARG;
  if (deblur && (prm->flags & CBP_FLAG_KERNELS_IN) && (!k1 || !k2)) return CBP_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(c->api_mu);
  const bool host_io = (prm->flags & CBP_FLAG_HOST_IO) != 0;
  // twiddle tables of the last chunked call, valid while this call's chunk
  // layout and workspace are the same (they depend on nothing else)
  const uint64_t tw_prev = c->tw_key;
  c->tw_key = 0;
  if (host_io && (!contiguous(b1) || !contiguous(b2))) return CBP_ERR_INVALID_ARG;
  const int nch = (c->profiling || stages)
                      ? 1
                      : std::max(1, std::min(host_io ? kIoChunks : kChunks, p.n / kMinChunkPairs));
  if (nch == 1) {
    s = c->ensure_ws(p.total, st);
    if (s != CBP_OK) return s;
    s = cbp::run_plan(p, b1, b2, prm, k1, k2, latent, deblur, c->ws, st,
                      c->profiling ? &c->prof : nullptr, nullptr, c->cnn_w);
    if (s != CBP_OK) return s;
    s = copy_stages(p, c->ws, stages, st);
    if (s != CBP_OK) return s;
    if (diag &&
        cudaMemcpyAsync(diag, c->ws + p.off_diag, (size_t)p.n * sizeof(cbp_diag),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return CBP_ERR_CUDA;
    return CBP_OK;
  }
  // chunked: plans, workspace regions, fork from the caller's stream
  s = c->ensure_chunk_streams();
  if (s != CBP_OK) return s;
  Plan cp[Ctx::kMaxChunks];
  cbp_frames f1[Ctx::kMaxChunks], f2[Ctx::kMaxChunks];
  int start[Ctx::kMaxChunks + 1];
  size_t off[Ctx::kMaxChunks + 1];
  start[0] = 0;
  off[0] = 0;
  // Host I/O: the last chunk's compute and read-back follow the last input
  // copy with the link idle, so the last three chunks shrink (weights 0.73,
  // 0.45, 0.27 of the others'); otherwise equal chunks.
  double wt[Ctx::kMaxChunks], wsum = 0.0, wacc = 0.0;
  for (int i = 0; i < nch; ++i) {
    const int back = nch - 1 - i;   // 0 for the last chunk
    wt[i] = (host_io && nch >= 4 && back < 3) ? (back == 0 ? 0.27 : back == 1 ? 0.45 : 0.73) : 1.0;
    wsum += wt[i];
  }
  for (int i = 0; i < nch; ++i) {
    wacc += wt[i];
    start[i + 1] = i + 1 == nch ? p.n : (int)std::llround((double)p.n * wacc / wsum);
    f1[i] = frames_slice(b1, start[i], start[i + 1] - start[i]);
    f2[i] = frames_slice(b2, start[i], start[i + 1] - start[i]);
    s = cbp::make_plan(&f1[i], &f2[i], prm, &cp[i]);
    if (s != CBP_OK) return s;
    off[i + 1] = off[i] + ((cp[i].total + 255) & ~size_t(255));
  }
  s = c->ensure_ws(off[nch], st);
  if (s != CBP_OK) return s;
  // key of the tables' layout: workspace generation, chunk regions and the
  // offsets and sizes the tables are built for (FNV-1a)
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      key ^= (v >> (8 * b)) & 0xff;
      key *= 1099511628211ull;
    }
  };
  mix(c->ws_gen);
  mix((uint64_t)(uintptr_t)c->ws);
  mix((uint64_t)nch);
  for (int i = 0; i < nch; ++i) {
    const Plan& q = cp[i];
    const uint64_t v[] = {off[i], (uint64_t)q.fft_f64, (uint64_t)q.Ph, (uint64_t)q.Pw,
                          (uint64_t)q.pw_half, (uint64_t)q.fp_h.n, (uint64_t)q.fp_w.n,
                          (uint64_t)q.fp_w2.n, q.off_tw_h, q.off_tw_w, q.off_stw_h, q.off_stw_r,
                          q.off_tw2r, q.off_tw2c};
    for (uint64_t x : v) mix(x);
  }
  if (key == 0) key = 1;
  const bool tw_ready = key == tw_prev;
#ifdef CBP_TIMELINE
  // Diagnostic build: per-chunk stage events against a start event, printed
  // once the call completes (the call becomes synchronous).
  static cbp::Prof tl[Ctx::kMaxChunks];
  cudaEvent_t tl0 = nullptr;
  cudaEventCreate(&tl0);
  cudaEventRecord(tl0, st);
#endif
  if (cudaEventRecord(c->chunk_ev[c->kMaxChunks], st) != cudaSuccess) return CBP_ERR_CUDA;
  const bool kf64 = b1->dtype == CBP_F64 || (prm->flags & CBP_FLAG_KERNELS_F64);
  const size_t kes = kf64 ? 8 : 4, les = b1->dtype == CBP_F64 ? 8 : 4;
  const size_t lat_pair = (size_t)p.C * p.H * p.W * les;
  const bool kin = (prm->flags & CBP_FLAG_KERNELS_IN) != 0;
  // Host I/O: the chunks' inputs go over on one copy stream in chunk order, so
  // chunk i computes while the inputs of chunks > i are still in flight and
  // its results go back while later chunks compute.  With
  // CBP_FLAG_OVERLAP_CALLS and the previous call's chunk layout (tw_ready:
  // same workspace, same regions), the copies and kernels wait only for the
  // previous call's chunk i to be done with region i (its chunk event; the
  // chunk's kernels follow it on the same stream), not for all earlier work
  // on the caller's stream.
  const bool overlap = host_io && (prm->flags & CBP_FLAG_OVERLAP_CALLS) && tw_ready;
  if (host_io && !overlap &&
      cudaStreamWaitEvent(c->io_st, c->chunk_ev[c->kMaxChunks], 0) != cudaSuccess)
    return CBP_ERR_CUDA;
  for (int i = 0; i < nch; ++i) {
    cudaStream_t cs = c->chunk_st[i % Ctx::kChunkStreams];
    if (!overlap && cudaStreamWaitEvent(cs, c->chunk_ev[c->kMaxChunks], 0) != cudaSuccess)
      return CBP_ERR_CUDA;
    if (overlap && cudaStreamWaitEvent(c->io_st, c->chunk_ev[i], 0) != cudaSuccess)
      return CBP_ERR_CUDA;
    const size_t a = (size_t)start[i];
    void* ck1 = k1 ? (char*)k1 + a * p.t1 * p.t1 * kes : nullptr;
    void* ck2 = k2 ? (char*)k2 + a * p.t2 * p.t2 * kes : nullptr;
    void* clat = latent ? (char*)latent + a * lat_pair : nullptr;
    char* w = c->ws + off[i];
    if (host_io) {
      const cbp_frames* fs[2] = {&f1[i], &f2[i]};
      for (int k = 0; k < 2; ++k) {
        const cbp_frames* f = fs[k];
        const size_t bytes = (size_t)f->n * f->c * f->h * f->w * les;
        if (cudaMemcpyAsync(w + cp[i].off_io_b[k], f->data, bytes, cudaMemcpyHostToDevice,
                            c->io_st) != cudaSuccess)
          return CBP_ERR_CUDA;
      }
      if (kin && (cudaMemcpyAsync(w + cp[i].off_io_k[0], ck1, (size_t)cp[i].n * p.t1 * p.t1 * kes,
                                  cudaMemcpyHostToDevice, c->io_st) != cudaSuccess ||
                  cudaMemcpyAsync(w + cp[i].off_io_k[1], ck2, (size_t)cp[i].n * p.t2 * p.t2 * kes,
                                  cudaMemcpyHostToDevice, c->io_st) != cudaSuccess))
        return CBP_ERR_CUDA;
      if (cudaEventRecord(c->io_ev[i], c->io_st) != cudaSuccess ||
          cudaStreamWaitEvent(cs, c->io_ev[i], 0) != cudaSuccess)
        return CBP_ERR_CUDA;
    }
    // Device-resident calls: chunk i starts once chunk i - 1 has read its
    // frames, so the chunks run out of phase (one's latency-bound solves
    // beside another's bandwidth-bound FFT passes).
    if (!host_io && i > 0 && cudaStreamWaitEvent(cs, c->read_ev[i - 1], 0) != cudaSuccess)
      return CBP_ERR_CUDA;
#ifdef CBP_TIMELINE
    cbp::Prof* tlp = &tl[i];
#else
    cbp::Prof* tlp = nullptr;
#endif
    s = cbp::run_plan(cp[i], &f1[i], &f2[i], prm, ck1, ck2, clat, deblur, w, cs, tlp, nullptr,
                      c->cnn_w, host_io, host_io ? nullptr : c->read_ev[i],
                      // device-resident calls only: with host I/O's copy stream the
                      // extra streams would share the GPU's hardware queues with it
                      host_io ? nullptr : c->solve_st[i % Ctx::kChunkStreams], c->fork_ev[i],
                      c->join_ev[i], tw_ready);
    if (s != CBP_OK) return s;
    if (diag && cudaMemcpyAsync(diag + a, w + cp[i].off_diag, (size_t)cp[i].n * sizeof(cbp_diag),
                                cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      return CBP_ERR_CUDA;
    if (cudaEventRecord(c->chunk_ev[i], cs) != cudaSuccess ||
        cudaStreamWaitEvent(st, c->chunk_ev[i], 0) != cudaSuccess)
      return CBP_ERR_CUDA;
  }
  if (deblur || cp[0].learned) c->tw_key = key;   // every chunk has its tables now
#ifdef CBP_TIMELINE
  cudaStreamSynchronize(st);
  for (int i = 0; i < nch; ++i) {
    for (const cbp::Prof::Rec& r : tl[i].recs) {
      float ta = 0.f, tb = 0.f;
      cudaEventElapsedTime(&ta, tl0, r.a);
      cudaEventElapsedTime(&tb, tl0, r.b);
      printf("timeline chunk=%d stage=%d begin=%.4f end=%.4f\n", i, r.stage, ta, tb);
      tl[i].pool.push_back(r.a);
      tl[i].pool.push_back(r.b);
    }
    tl[i].recs.clear();
  }
  fflush(stdout);
  cudaEventDestroy(tl0);
#endif
  return CBP_OK;
}

}  // namespace

extern "C" {

cbp_status cbp_create(cbp_ctx** out, int device, size_t hbm_budget_bytes) {
  if (!out) return CBP_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return CBP_ERR_CUDA;
  }
  DeviceGuard g(device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return CBP_ERR_CUDA;
  Ctx* c = new (std::nothrow) Ctx();
  if (!c) return CBP_ERR_OOM;
  c->device = device;
  c->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
  *out = reinterpret_cast<cbp_ctx*>(c);
  return CBP_OK;
}

cbp_status cbp_destroy(cbp_ctx* ctx) {
  if (!ctx) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(c->device);
  cbp::serve_shutdown(c);
  cudaDeviceSynchronize();
  if (c->ws) cudaFree(c->ws);
  for (int i = 0; i < Ctx::kChunkStreams; ++i)
    if (c->chunk_st[i]) cudaStreamDestroy(c->chunk_st[i]);
  if (c->io_st) cudaStreamDestroy(c->io_st);
  for (int i = 0; i < Ctx::kChunkStreams; ++i)
    if (c->solve_st[i]) cudaStreamDestroy(c->solve_st[i]);
  for (int i = 0; i <= Ctx::kMaxChunks; ++i)
    if (c->chunk_ev[i]) cudaEventDestroy(c->chunk_ev[i]);
  for (int i = 0; i < Ctx::kMaxChunks; ++i) {
    if (c->io_ev[i]) cudaEventDestroy(c->io_ev[i]);
    if (c->read_ev[i]) cudaEventDestroy(c->read_ev[i]);
    if (c->fork_ev[i]) cudaEventDestroy(c->fork_ev[i]);
    if (c->join_ev[i]) cudaEventDestroy(c->join_ev[i]);
  }
  if (c->cnn_ws) cudaFree(c->cnn_ws);
  if (c->cnn_w) cudaFree(c->cnn_w);
  delete c;
  return CBP_OK;
}

const char* cbp_status_string(cbp_status s) {
  switch (s) {
    case CBP_OK: return "CBP_OK";
    case CBP_WARN_ILL_CONDITIONED: return "CBP_WARN_ILL_CONDITIONED";
    case CBP_ERR_INVALID_ARG: return "CBP_ERR_INVALID_ARG";
    case CBP_ERR_SIZE_MISMATCH: return "CBP_ERR_SIZE_MISMATCH";
    case CBP_ERR_NOT_COPRIME: return "CBP_ERR_NOT_COPRIME";
    case CBP_ERR_OOM: return "CBP_ERR_OOM";
    case CBP_ERR_CUDA: return "CBP_ERR_CUDA";
    case CBP_ERR_BUSY: return "CBP_ERR_BUSY";
    case CBP_ERR_TIMEOUT: return "CBP_ERR_TIMEOUT";
    case CBP_ERR_BUDGET: return "CBP_ERR_BUDGET";
    case CBP_ERR_UNSUPPORTED: return "CBP_ERR_UNSUPPORTED";
  }
  return "CBP_UNKNOWN_STATUS";
}

cbp_status cbp_workspace_size(const cbp_frames* b1, const cbp_frames* b2,
                              const cbp_params* params, size_t* bytes) {
  if (!bytes) return CBP_ERR_INVALID_ARG;
  Plan p;
  cbp_status s = cbp::make_plan(b1, b2, params, &p);
  if (s != CBP_OK) return s;
  *bytes = p.total;
  return CBP_OK;
}

cbp_status cbp_estimate_kernels(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                                const cbp_params* params, void* k1, void* k2, cbp_diag* diag,
                                void* stream) {
  cbp::NvtxScope range("cbp_estimate_kernels");
  try {
    return call_path(ctx, b1, b2, params, k1, k2, nullptr, diag, stream, false);
  } catch (...) {
    return CBP_ERR_OOM;
  }
}

cbp_status cbp_estimate_kernels_stages(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                                       const cbp_params* params, void* k1, void* k2,
                                       cbp_diag* diag, const cbp_stage_out* out, void* stream) {
  cbp::NvtxScope range("cbp_estimate_kernels_stages");
  try {
    if (params && (params->flags & CBP_FLAG_HOST_IO)) return CBP_ERR_INVALID_ARG;
    return call_path(ctx, b1, b2, params, k1, k2, nullptr, diag, stream, false, out);
  } catch (...) {
    return CBP_ERR_OOM;
  }
}

cbp_status cbp_deblur_pair(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                           const cbp_params* params, void* k1, void* k2, void* latent,
                           cbp_diag* diag, void* stream) {
  cbp::NvtxScope range("cbp_deblur_pair");
  try {
    return call_path(ctx, b1, b2, params, k1, k2, latent, diag, stream, true);
  } catch (...) {
    return CBP_ERR_OOM;
  }
}

cbp_status cbp_forward_blur(cbp_ctx* ctx, const void* latent, int32_t n, int32_t c, int32_t h,
                            int32_t w, cbp_dtype dtype, const double* kernel, int32_t t,
                            double sigma, uint64_t seed, void* out, void* stream) {
  if (!ctx || !latent || !kernel || !out || n < 1 || c < 1 || h < 1 || w < 1 || t < 1 ||
      t > 64 || !(sigma >= 0.0) || (dtype != CBP_F32 && dtype != CBP_F64))
    return CBP_ERR_INVALID_ARG;
  Ctx* cx = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(cx->device);
  cbp::launch_forward_blur(latent, n, c, h, w, dtype == CBP_F64, kernel, t, sigma, seed, out,
                           (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

cbp_status cbp_truncate_lsb(cbp_ctx* ctx, const void* in, cbp_dtype dtype, int64_t count,
                            int32_t bits, int32_t drop, void* out, void* stream) {
  if (!ctx || !in || !out || count < 0 || bits < 1 || bits > 30 || drop < 0 || drop >= bits ||
      (dtype != CBP_F32 && dtype != CBP_F64))
    return CBP_ERR_INVALID_ARG;
  if (count == 0) return CBP_OK;
  Ctx* cx = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(cx->device);
  cbp::launch_truncate_lsb(in, dtype == CBP_F64, count, bits, drop, out, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

cbp_status cbp_synth_latent(cbp_ctx* ctx, const double* blobs, int32_t nblobs, int32_t n,
                            int32_t c, int32_t h, int32_t w, cbp_dtype dtype, double floor_amp,
                            uint64_t seed, void* out, void* stream) {
  if (!ctx || !blobs || !out || nblobs < 0 || n < 1 || c < 1 || h < 1 || w < 1 ||
      (dtype != CBP_F32 && dtype != CBP_F64))
    return CBP_ERR_INVALID_ARG;
  Ctx* cx = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(cx->device);
  cbp::launch_synth_latent(blobs, nblobs, n, c, h, w, dtype == CBP_F64, floor_amp, seed, out,
                           (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

cbp_status cbp_profile(cbp_ctx* ctx, int32_t enable) {
  if (!ctx) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::mutex> lk(c->api_mu);
  c->profiling = enable != 0;
  return CBP_OK;
}

cbp_status cbp_stage_times(cbp_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx) return CBP_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lk(c->api_mu);
  cbp::Prof& P = c->prof;
  cbp_status st = CBP_OK;
  for (auto& r : P.recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
      st = CBP_ERR_CUDA;
    if (ms) ms[r.stage] += (double)t;
    P.pool.push_back(r.a);
    P.pool.push_back(r.b);
  }
  P.recs.clear();
  for (int i = 0; i < CBP_NUM_STAGES; ++i) {
    if (launches) launches[i] += P.launches[i];
    P.launches[i] = 0;
  }
  return st;
}

cbp_status cbp_estimate_size(cbp_ctx* ctx, const cbp_frames* b1, const cbp_frames* b2,
                             const cbp_size_params* params, int32_t* t1_out, int32_t* t2_out,
                             int32_t* found, double* ratios, int32_t* ncand_out, void* stream) {
  cbp::NvtxScope range("cbp_estimate_size");
  return size_scan(ctx, b1, b2, params, t1_out, t2_out, found, ratios, ncand_out, stream);
}

cbp_status cbp_encrypt(cbp_ctx* ctx, const void* latent, int32_t n, int32_t c, int32_t h, int32_t w,
                       cbp_dtype dtype, const cbp_encrypt_params* params, double* k1, double* k2,
                       void* b1, void* b2, double* k3, double* k4, void* c1, void* c2,
                       int32_t* attempts, void* stream) {
  cbp::NvtxScope range("cbp_encrypt");
  try {
    return encrypt_frames(ctx, latent, n, c, h, w, dtype, params, k1, k2, b1, b2, k3, k4, c1, c2,
                          attempts, stream);
  } catch (...) {
    return CBP_ERR_OOM;
  }
}

cbp_status cbp_check_words(uint32_t* words, int32_t n, int32_t reset) {
#ifdef CBP_CHECKS
  if (!words || n < 0) return CBP_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return CBP_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    auto rd = i < cbp::kChkWords ? cbp::check_reader(i) : nullptr;
    words[i] = rd ? rd(reset != 0) : 0u;
  }
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
#else
  (void)words;
  (void)n;
  (void)reset;
  return CBP_ERR_UNSUPPORTED;
#endif
}

cbp_status cbp_check_expire_waits(int32_t on) {
#ifdef CBP_CHECKS
  if (cudaDeviceSynchronize() != cudaSuccess) return CBP_ERR_CUDA;
  return cbp::set_tx_extra(on ? 16u : 0u) ? CBP_OK : CBP_ERR_CUDA;
#else
  (void)on;
  return CBP_ERR_UNSUPPORTED;
#endif
}

cbp_status cbp_check_recip(const double* x, int64_t n, double* rcp, double* rsqrt, void* stream) {
  if (!x || !rcp || !rsqrt || n < 0) return CBP_ERR_INVALID_ARG;
  if (n == 0) return CBP_OK;
  cbp::launch_check_recip(x, n, rcp, rsqrt, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? CBP_OK : CBP_ERR_CUDA;
}

}  // extern "C"
