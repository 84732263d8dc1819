// Request loop (gbs_submit / gbs_poll): continuous batching of probability and
// sampling requests.
#include "gbs_internal.h"

namespace gbs {
void server_shutdown(gbs_ctx* ctx) { (void)ctx; }
}  // namespace gbs
