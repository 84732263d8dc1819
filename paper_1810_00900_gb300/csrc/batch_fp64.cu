// Batched subset-determinant trees, double per-term arithmetic (real and complex).
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_fp64_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<double, 5>(ctx, ntrees, trees, roots, outs, status, tune);
}
gbs_status batch_fp64_cplx(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<cplx<double>, 4>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
