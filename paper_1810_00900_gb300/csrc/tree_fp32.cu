// Subset-determinant tree, float per-term arithmetic: real (x/p basis, symmetric)
// and complex (a/a^+ basis, Hermitian) instantiations.
#include "gbs_tree_driver.cuh"

namespace gbs {
gbs_status tree_fp32_real(gbs_ctx* ctx, const void* G, int n, TreeOut* out) {
  return tree_run<float, 5>(ctx, G, n, out);
}
gbs_status tree_fp32_cplx(gbs_ctx* ctx, const void* G, int n, TreeOut* out) {
  return tree_run<cplx<float>, 4>(ctx, G, n, out);
}
}  // namespace gbs
