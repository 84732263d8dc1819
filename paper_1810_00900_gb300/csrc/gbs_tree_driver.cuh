// Host driver of the subset-determinant tree for one element type.
// Included by tree_fp64.cu, tree_dd.cu, tree_td.cu and tree_fp32.cu so that
// each precision compiles in its own translation unit (in parallel).
#pragma once
#include <algorithm>
#include <string>

#include "gbs_internal.h"
#include "gbs_tree.cuh"

namespace gbs {

template <class E> struct root_src { typedef double type; };
template <class T> struct root_src<cplx<T>> { typedef cplx<double> type; };

template <class T> GBS_HD T conv_from64(double x) { return from_double<T>(x); }
template <class E> GBS_HD E conv_entry(const typename root_src<E>::type& x);
template <> GBS_HD double conv_entry<double>(const double& x) { return x; }
template <> GBS_HD float conv_entry<float>(const double& x) { return (float)x; }
template <> GBS_HD dd conv_entry<dd>(const double& x) { return dd_make(x); }
template <> GBS_HD td conv_entry<td>(const double& x) { return td_make(x); }
template <> GBS_HD cplx<double> conv_entry<cplx<double>>(const cplx<double>& x) { return x; }
template <> GBS_HD cplx<float> conv_entry<cplx<float>>(const cplx<double>& x) { return {(float)x.re, (float)x.im}; }
template <> GBS_HD cplx<dd> conv_entry<cplx<dd>>(const cplx<double>& x) { return {dd_make(x.re), dd_make(x.im)}; }
template <> GBS_HD cplx<td> conv_entry<cplx<td>>(const cplx<double>& x) { return {td_make(x.re), td_make(x.im)}; }

template <class E>
__global__ void tree_root_kernel(const typename root_src<E>::type* __restrict__ g, int nent, E* __restrict__ root,
                                 typename real_of<E>::type* __restrict__ s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nent) root[i] = conv_entry<E>(g[i]);
  if (i == 0) s[0] = from_double<typename real_of<E>::type>(1.0);
}

template <class E, int Q>
static void launch_leaf(int blocks, cudaStream_t st, const E* nodes, const typename real_of<E>::type* s,
                        long long count, int depth,
                        Partial<typename acc_traits<typename real_of<E>::type>::Red>* parts, int* status) {
  tree_leaf_kernel<E, Q><<<blocks, 128, 0, st>>>(nodes, s, count, depth, parts, status);
}

template <class E, int QMAX>
static void launch_leaf_q(int Q, int blocks, cudaStream_t st, const E* nodes,
                          const typename real_of<E>::type* s, long long count, int depth,
                          Partial<typename acc_traits<typename real_of<E>::type>::Red>* parts, int* status) {
  if constexpr (QMAX >= 1) {
    if (Q == QMAX) {
      launch_leaf<E, QMAX>(blocks, st, nodes, s, count, depth, parts, status);
      return;
    }
    launch_leaf_q<E, (QMAX > 1 ? QMAX - 1 : 0)>(Q, blocks, st, nodes, s, count, depth, parts, status);
  }
}

// Largest per-level node storage (entries) of a tree over n modes with Q leaf levels.
inline size_t tree_level_entries(int n, int Q) {
  size_t best = 0;
  for (int l = 0; l <= n - Q; ++l) {
    const size_t count = (size_t)1 << l;
    const int q = n - l;
    best = std::max(best, count * (size_t)sym(2 * q));
  }
  return best;
}

template <class E, int QMAX>
gbs_status tree_run(gbs_ctx* ctx, const void* groot, int n, TreeOut* out) {
  typedef typename real_of<E>::type T;
  typedef typename acc_traits<T>::Red Red;
  if (n < 1 || n > 40) return set_error(ctx, GBS_EINVAL, "tree: n must be in [1, 40]");
  const int Q = std::min(n, QMAX);
  const int depth = n - Q;
  const long long leaves = 1LL << depth;
  const size_t ent = tree_level_entries(n, Q);
  const int blocks = (int)((leaves + 127) / 128);
  gbs_status st;
  if ((st = dev_reserve(ctx, ctx->lvl[0], ent * sizeof(E)))) return st;
  if ((st = dev_reserve(ctx, ctx->lvl[1], ent * sizeof(E)))) return st;
  if ((st = dev_reserve(ctx, ctx->sbuf[0], (size_t)leaves * sizeof(T)))) return st;
  if ((st = dev_reserve(ctx, ctx->sbuf[1], (size_t)leaves * sizeof(T)))) return st;
  if ((st = dev_reserve(ctx, ctx->partials, (size_t)blocks * sizeof(Partial<Red>)))) return st;
  if ((st = dev_reserve(ctx, ctx->status, sizeof(int)))) return st;
  cudaStream_t s = ctx->stream;
  int* status = (int*)ctx->status.ptr;
  if ((st = check_cuda(ctx, cudaMemsetAsync(status, 0, sizeof(int), s), "memset status"))) return st;

  E* lv[2] = {(E*)ctx->lvl[0].ptr, (E*)ctx->lvl[1].ptr};
  T* sv[2] = {(T*)ctx->sbuf[0].ptr, (T*)ctx->sbuf[1].ptr};
  const int nent = sym(2 * n);
  tree_root_kernel<E><<<(nent + 255) / 256, 256, 0, s>>>((const typename root_src<E>::type*)groot, nent, lv[0], sv[0]);
  count_launch(ctx);
  int cur = 0;
  for (int l = 0; l < depth; ++l) {
    const long long count = 1LL << l;
    const int q = n - l;
    const long long threads = count * (2 * q - 2);
    const int tpb = 256;
    const long long nb = (threads + tpb - 1) / tpb;
    tree_level_kernel<E><<<(unsigned)nb, tpb, 0, s>>>(lv[cur], sv[cur], count, q, lv[cur ^ 1], sv[cur ^ 1], status);
    count_launch(ctx);
    cur ^= 1;
  }
  Partial<Red>* parts = (Partial<Red>*)ctx->partials.ptr;
  if (ctx->timing) {
    if (!ctx->leaf_timer.start) {
      cudaEventCreate(&ctx->leaf_timer.start);
      cudaEventCreate(&ctx->leaf_timer.stop);
    }
    cudaEventRecord(ctx->leaf_timer.start, s);
  }
  launch_leaf_q<E, QMAX>(Q, blocks, s, lv[cur], sv[cur], leaves, depth, parts, status);
  count_launch(ctx);
  if (ctx->timing) {
    cudaEventRecord(ctx->leaf_timer.stop, s);
    ctx->leaf_timer.pending = true;
  }
  tree_final_kernel<Red><<<1, 256, 0, s>>>(parts, blocks, out);
  count_launch(ctx);
  return check_cuda(ctx, cudaGetLastError(), "tree launch");
}

}  // namespace gbs
