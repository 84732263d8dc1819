// Batched subset-determinant trees, fixed-point (160 fraction bits) per-term arithmetic (real basis).
#include "gbs_fx.cuh"
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_fx_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                         int* status, const BatchTune& tune) {
  return batch_run<fx, 3>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
