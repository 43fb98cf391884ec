// Batched solving and the continuous-batching server (entry points of
// include/lp.h).  Placeholder until the segmented persistent kernel lands.
#include "lp_internal.h"

namespace gb300lp {
void set_last_error(const std::string &m);
}

extern "C" {
int lp_server_create(size_t, const lp_device_ctx *, const lp_solve_opts *, int32_t,
                     lp_server **out) {
  if (out) *out = nullptr;
  gb300lp::set_last_error("batched server not available in this build");
  return LP_ERR_STATE;
}
int lp_batch_submit(lp_server *, lp_problem *, uint64_t *) { return LP_ERR_STATE; }
int lp_batch_poll(lp_server *, uint64_t, lp_result *, double *, double *) { return LP_ERR_STATE; }
int lp_server_pump(lp_server *, int32_t) { return LP_ERR_STATE; }
int lp_batch_cancel(lp_server *, uint64_t) { return LP_ERR_STATE; }
int lp_server_stats(const lp_server *, int64_t *) { return LP_ERR_STATE; }
void lp_server_destroy(lp_server *) {}
}
