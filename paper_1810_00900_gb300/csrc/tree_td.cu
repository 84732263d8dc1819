// Subset-determinant tree, td per-term arithmetic: real (x/p basis, symmetric)
// and complex (a/a^+ basis, Hermitian) instantiations.
#include "gbs_tree_driver.cuh"

namespace gbs {
gbs_status tree_td_real(gbs_ctx* ctx, const void* G, int n, TreeOut* out) {
  return tree_run<td, 3>(ctx, G, n, out);
}
gbs_status tree_td_cplx(gbs_ctx* ctx, const void* G, int n, TreeOut* out) {
  return tree_run<cplx<td>, 2>(ctx, G, n, out);
}
}  // namespace gbs
