// Batched subset-determinant trees, float per-term arithmetic (real and complex).
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_fp32_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<float, 5>(ctx, ntrees, trees, roots, outs, status, tune);
}
gbs_status batch_fp32_cplx(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<cplx<float>, 4>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
