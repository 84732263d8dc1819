// Batched subset-determinant trees, narrow fixed-point per-term arithmetic
// (128 fraction bits, real basis).
#include "gbs_fx.cuh"
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_fxn_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<fxn4, 3>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
