// Serving loop: placeholder until the continuous-batching server lands.
#include "bqc_internal.h"

extern "C" {
int bqc_serve_create(bqc_ctx *, const bqc_serve_opts *, bqc_server **out) {
  if (out) *out = nullptr;
  return BQC_E_UNSUPPORTED;
}
int bqc_serve_submit(bqc_server *, const bqc_request *, uint64_t *) { return BQC_E_UNSUPPORTED; }
int bqc_serve_poll(bqc_server *, uint64_t, bqc_serve_result *) { return BQC_E_UNSUPPORTED; }
int bqc_serve_drain(bqc_server *, double) { return BQC_E_UNSUPPORTED; }
int bqc_serve_destroy(bqc_server *) { return BQC_E_UNSUPPORTED; }
size_t bqc_serve_footprint(int, int, int) { return 0; }
}
