// Batched subset-determinant trees, FP64 real basis with the last two levels of
// every tree evaluated as cancellation-free groups.
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_fp64p_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                            int* status, const BatchTune& tune) {
  return batch_run<double, 5, true>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
