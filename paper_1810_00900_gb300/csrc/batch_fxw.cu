// Batched subset-determinant trees, wide fixed-point per-term arithmetic (real basis).
#include "gbs_fx.cuh"
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_fxw_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<fxw, 3>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
