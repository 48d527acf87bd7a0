// Context object and serving-engine interface (internal).
#pragma once
#include <cuda_runtime.h>
#include <mutex>
#include <vector>
#include "cbp.h"
#include "cbp_internal.h"

namespace cbp {

struct ServeState;  // defined in cbp_serve.cu

// Request flags the serving engine does not take (it works on device buffers).
constexpr int kServeRejectFlags = CBP_FLAG_HOST_IO;

// Stage timing: events recorded around each stage of the synchronous API.
struct Prof {
  struct Rec { int stage; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int64_t launches[CBP_NUM_STAGES] = {};
  cudaEvent_t get();
  void begin(int stage, cudaStream_t st, cudaEvent_t* a);
  void end(int stage, cudaStream_t st, cudaEvent_t a, int nkernels);
};

struct Ctx {
  int device = 0;
  size_t budget = 0;          // bytes of device memory the context may hold
  size_t used = 0;            // bytes held now
  std::mutex mem_mu;          // guards used
  std::mutex api_mu;          // serialises the synchronous API's workspace use
  char* ws = nullptr;         // synchronous-API workspace
  size_t ws_size = 0;
  uint64_t ws_gen = 0;        // bumped whenever `ws` is replaced
  // FFT twiddle tables left in `ws` by the last chunked call: a key of the
  // workspace and the chunks' table layout (0: none valid)
  uint64_t tw_key = 0;
  ServeState* serve = nullptr;
  bool profiling = false;
  Prof prof;
  // internal streams and fork/join events of chunked synchronous calls
  static constexpr int kMaxChunks = 8;        // chunks of one call
  static constexpr int kChunkStreams = 4;     // compute streams they rotate over
  cudaStream_t chunk_st[kChunkStreams] = {};
  cudaStream_t io_st = nullptr;               // host-to-device copies of host-I/O calls, in order
  cudaEvent_t chunk_ev[kMaxChunks + 1] = {};
  cudaEvent_t io_ev[kMaxChunks] = {};
  cudaEvent_t read_ev[kMaxChunks] = {};      // chunk i has read its frames (row pass done)
  // high-priority streams of the chunks' latency-bound solves: their blocks
  // are placed before the pending FFT blocks of the other chunks
  cudaStream_t solve_st[kChunkStreams] = {};
  cudaEvent_t fork_ev[kMaxChunks] = {};
  cudaEvent_t join_ev[kMaxChunks] = {};
  bool chunk_ready = false;
  cbp_status ensure_chunk_streams();
  std::mutex serve_mu;        // guards creation of `serve`
  float* cnn_w = nullptr;     // learned-path weights (cbp_learned_load)
  char* cnn_ws = nullptr;     // workspace of the standalone network calls
  size_t cnn_ws_size = 0;

  bool reserve(size_t bytes);
  void release(size_t bytes);
  cbp_status ensure_ws(size_t bytes, cudaStream_t st);
  cbp_status ensure_cnn_ws(size_t bytes, cudaStream_t st);
};

cbp_status run_plan(const Plan& p, const cbp_frames* b1, const cbp_frames* b2,
                    const cbp_params* prm, void* k1, void* k2, void* latent, bool deblur,
                    char* wsp, cudaStream_t st, Prof* prof = nullptr,
                    const PtrTables* tabs = nullptr, const float* cnn_w = nullptr,
                    bool h2d_done = false,    // host I/O: inputs already copied by the caller
                    cudaEvent_t after_read = nullptr,   // recorded once the frames are read
                    // estimation kernels on `solve` (forked from and joined to st by
                    // the two events) when given
                    cudaStream_t solve = nullptr, cudaEvent_t fork = nullptr,
                    cudaEvent_t join = nullptr,
                    bool tw_ready = false);   // the twiddle tables are already in wsp
void serve_shutdown(Ctx* c);

}  // namespace cbp
