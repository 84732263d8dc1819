// Batched subset-determinant trees, td per-term arithmetic (real and complex).
#include "gbs_batch_driver.cuh"

namespace gbs {
gbs_status batch_td_real(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<td, 3>(ctx, ntrees, trees, roots, outs, status, tune);
}
gbs_status batch_td_cplx(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots, TreeOut* outs,
                          int* status, const BatchTune& tune) {
  return batch_run<cplx<td>, 2>(ctx, ntrees, trees, roots, outs, status, tune);
}
}  // namespace gbs
