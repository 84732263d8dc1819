// Batched subset-determinant trees, dd per-term arithmetic (real and complex).
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_dd_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<dd, 4>(ctx, ntrees, trees, roots, outs, status, tune);
}
gbs_status batch_dd_cplx(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<cplx<dd>, 3>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
