// Serving engine (continuous batching) -- placeholder until implemented.
#include "cbp_serve.h"

namespace cbp {
void serve_shutdown(Ctx*) {}
}  // namespace cbp

extern "C" {
cbp_status cbp_stream_submit(cbp_ctx*, const cbp_frames*, const cbp_frames*, const cbp_params*,
                             void*, void*, void*, uint64_t*) {
  return CBP_ERR_UNSUPPORTED;
}
cbp_status cbp_stream_poll(cbp_ctx*, uint64_t, int32_t, cbp_diag*) { return CBP_ERR_UNSUPPORTED; }
cbp_status cbp_stream_stats(cbp_ctx*, uint64_t*, double*, double*, int32_t) {
  return CBP_ERR_UNSUPPORTED;
}
}
