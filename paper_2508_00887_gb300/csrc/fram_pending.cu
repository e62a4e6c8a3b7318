// Entry points whose GPU paths are being brought up.  Until then they return
// FRAM_ERR_INVALID with a message rather than computing anything on the host.
#include "fram_ctx.h"

namespace fram {

void serve_shutdown(fram_ctx*) {}

}  // namespace fram

extern "C" {

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
