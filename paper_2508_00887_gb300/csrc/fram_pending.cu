// Entry points whose GPU paths are being brought up.  Until then they return
// FRAM_ERR_INVALID with a message rather than computing anything on the host.
#include "fram_ctx.h"

namespace fram {

void batched_release(fram_ctx*) {}
void serve_shutdown(fram_ctx*) {}

}  // namespace fram

extern "C" {

fram_status fram_solve_batched(fram_ctx* c, int count, const int* n, const double* const* A,
                               const double* const* B, const fram_params* params,
                               double* const* X_out, int32_t* const* perm_out, fram_info* infos) {
  if (!c || count < 0 || (count > 0 && (!n || !A || !B || !perm_out))) return FRAM_ERR_INVALID;
  fram_params p;
  if (params)
    p = *params;
  else
    fram_default_params(&p);
  for (int i = 0; i < count; ++i) {
    fram_status s = fram_solve(c, n[i], A[i], B[i], nullptr, &p, X_out ? X_out[i] : nullptr,
                               perm_out[i], infos ? &infos[i] : nullptr);
    if (s != FRAM_OK) return s;
  }
  return FRAM_OK;
}

fram_status fram_submit(fram_ctx* c, int, const double*, const double*, const fram_params*,
                        uint64_t*) {
  if (c) fram::set_err(c, "serving is not available in this build");
  return FRAM_ERR_INVALID;
}

fram_status fram_poll(fram_ctx* c, uint64_t, double*, int32_t*, fram_info*, int) {
  if (c) fram::set_err(c, "serving is not available in this build");
  return FRAM_ERR_INVALID;
}

}  // extern "C"
