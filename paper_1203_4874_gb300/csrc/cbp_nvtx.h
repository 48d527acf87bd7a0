// NVTX ranges around the library's entry points and the stages of a call, for
// timeline tools (Nsight Systems shows them on the calling thread, with the
// kernels each range enqueued).  Header-only NVTX 3: without a tool attached
// a range costs a load and a branch.  -DCBP_NO_NVTX compiles them out.
#pragma once
#ifndef CBP_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace cbp {

inline void nvtx_push(const char* name) {
#ifndef CBP_NO_NVTX
  nvtxRangePushA(name);
#else
  (void)name;
#endif
}
inline void nvtx_pop() {
#ifndef CBP_NO_NVTX
  nvtxRangePop();
#endif
}
// A range for the enclosing scope.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtx_push(name); }
  ~NvtxScope() { nvtx_pop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

}  // namespace cbp
