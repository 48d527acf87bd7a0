// Kernel estimation without any device allocation, for callers that may not
// allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates) at the
// point where they need the kernels: code running under a memory manager
// that owns every device allocation (a custom pool or a fixed arena), code
// that must not fail on allocation in the middle of a real-time video path,
// and code that has to keep its device footprint fixed from start-up.  This
// entry point runs the same estimation kernels as cbp_estimate_kernels, with
// their workspace placed in one file-scope device array of a fixed size
// (kNoAllocScratchBytes, 16 MiB: one 1080p RGB pair with 15x15 and 17x17
// kernels fits on either path) that every GPU loading the library holds until
// the process exits.
//
// Set-up: the array's device address belongs to the library's module in the
// current CUDA context.  It is looked up (cudaGetSymbolAddress, with the
// caller's device current) on every call made outside stream capture -- a
// host-side table lookup -- and remembered per (device, context), so a device
// reset or a context the caller pushed is picked up by the next such call.  A
// call made while its stream is capturing uses the address remembered for
// that device and context, so make the first call on a device (and the first
// after a device reset) before capturing any stream.  All calls share the one
// array and it keeps the previous call's contents: calls whose work overlaps
// on the GPU (different streams, or host threads without ordering) race on it
// and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <mutex>
#include "cbp.h"
#include "cbp_internal.h"

namespace cbp {
namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB
constexpr int kMaxContexts = 64;

static __device__ __align__(256) char g_noalloc_scratch[kNoAllocScratchBytes];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// The current driver context (nullptr when the driver entry point is not
// available; the device ordinal then keys the table alone).
void* current_context() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return (CtxGetCurrentFn)f;
  }();
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return (void*)c;
}

struct ScratchEntry {
  int dev;
  void* ctx;
  char* ptr;
};
std::mutex g_setup_mu;
ScratchEntry g_scratch[kMaxContexts] = {};
int g_nscratch = 0;

// Device address of the scratch array in the current device's context: looked
// up afresh outside stream capture, taken from the table during capture.
cbp_status scratch_for_current_context(cudaStream_t st, char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return CBP_ERR_CUDA;
  }
  void* ctx = current_context();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing =
      cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  if (capturing) cudaGetLastError();
  std::lock_guard<std::mutex> g(g_setup_mu);
  int slot = -1;
  for (int i = 0; i < g_nscratch; ++i)
    if (g_scratch[i].dev == dev && g_scratch[i].ctx == ctx) slot = i;
  if (capturing) {
    if (slot < 0) return CBP_ERR_CUDA;   // no address known for this context yet
    *out = g_scratch[slot].ptr;
    return CBP_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return CBP_ERR_CUDA;
  }
  if (slot < 0) {
    slot = g_nscratch < kMaxContexts ? g_nscratch++ : (int)(((uintptr_t)ctx >> 4) % kMaxContexts);
  }
  g_scratch[slot] = {dev, ctx, (char*)p};
  *out = (char*)p;
  return CBP_OK;
}

}  // namespace
}  // namespace cbp

extern "C" cbp_status cbp_estimate_kernels_noalloc(const cbp_frames* b1, const cbp_frames* b2,
                                                   const cbp_params* params, void* k1, void* k2,
                                                   cbp_diag* diag, void* stream) {
  using namespace cbp;
  if (!params || !k1 || !k2) return CBP_ERR_INVALID_ARG;
  if (params->flags & (CBP_FLAG_HOST_IO | CBP_FLAG_KERNELS_IN)) return CBP_ERR_INVALID_ARG;
  if (params->path == CBP_PATH_LEARNED) return CBP_ERR_UNSUPPORTED;   // needs the FFT workspace
  Plan p;
  cbp_status s = make_plan(b1, b2, params, &p);
  if (s != CBP_OK) return s;
  // The estimation buffers come first in the plan's layout; the deconvolution
  // buffers (from the twiddle tables on) are not used here.
  const size_t need = p.off_tw_h;
  if (need > kNoAllocScratchBytes) return CBP_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = nullptr;
  s = scratch_for_current_context(st, &ws);
  if (s != CBP_OK) return s;
  const int kf64 = b1->dtype == CBP_F64 || (params->flags & CBP_FLAG_KERNELS_F64);
  const FrameDesc d1 = frame_desc(b1, nullptr), d2 = frame_desc(b2, nullptr);
  // the non-finite flags accumulate with atomics: they must start at zero
  if (cudaMemsetAsync(ws + p.off_bad, 0, (size_t)p.n * sizeof(int), st) != cudaSuccess ||
      cudaMemsetAsync(ws + p.off_err, 0, sizeof(int), st) != cudaSuccess)
    return CBP_ERR_CUDA;
  launch_eval(p, d1, d2, ws, st);
  launch_sample_solve(p, ws, st);
  launch_scale_solve(p, ws, k1, k2, kf64, st);
  if (cudaGetLastError() != cudaSuccess) return CBP_ERR_CUDA;
  if (diag && cudaMemcpyAsync(diag, ws + p.off_diag, (size_t)p.n * sizeof(cbp_diag),
                              cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CBP_ERR_CUDA;
  return CBP_OK;
}
