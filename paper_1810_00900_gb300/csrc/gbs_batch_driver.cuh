// Host side of the batched tree engine: plan (segments, regions), upload, launches.
#pragma once
#include <algorithm>
#include <cstring>
#include <vector>

#include "gbs_batch.cuh"

namespace gbs {

// Append POD arrays to a byte blob at 16-byte aligned offsets.
struct Blob {
  std::vector<unsigned char> bytes;
  template <class X>
  size_t put(const std::vector<X>& v) {
    size_t off = (bytes.size() + 15) / 16 * 16;
    bytes.resize(off + v.size() * sizeof(X));
    if (!v.empty()) memcpy(bytes.data() + off, v.data(), v.size() * sizeof(X));
    return off;
  }
};


// PAIR: the last two levels of every tree as cancellation-free groups (FP64
// real basis; the tree's inc output then carries the whole Torontonian).
template <class E, int QMAX, bool PAIR = false>
gbs_status batch_run(gbs_ctx* ctx, int ntrees, const BatchTree* trees, const void* roots_dev, TreeOut* outs_dev,
                     int* status_dev, const BatchTune& tune) {
  typedef typename real_of<E>::type T;
  typedef typename scale_of<E>::type S;
  typedef typename acc_traits<T>::Red Red;
  if (ntrees <= 0) return GBS_OK;
  const int sub_e = std::max(0, std::min(tune.sub_e, 7));  // levels expanded inside a subtree CTA
  // ---------------- plan
  std::vector<int> Q(ntrees), depth(ntrees), dtop(ntrees), qroot(ntrees), emid(ntrees);
  std::vector<long long> region(ntrees), sreg(ntrees);
  long long region_total = 0, s_total = 0;
  int max_depth = 0, nmax = 0;
  for (int t = 0; t < ntrees; ++t) {
    const int n = trees[t].n;
    if (n < 1 || n > 40) return set_error(ctx, GBS_EINVAL, "batch tree size out of range");
    Q[t] = std::max(1, std::min(n, QMAX - tune.q_drop));
    qroot[t] = std::min(n, Q[t] + sub_e);
    depth[t] = n - qroot[t];  // levels above the leaf / subtree roots
    dtop[t] = std::min(depth[t], tune.d_top);
    emid[t] = std::min(depth[t] - dtop[t], std::max(0, std::min(tune.mid_e, 8)));
    long long biggest = 0;
    for (int l = dtop[t]; l <= depth[t]; ++l)
      biggest = std::max(biggest, (1LL << l) * (long long)sym(2 * (n - l)));
    region[t] = region_total;
    region_total += biggest;
    sreg[t] = s_total;
    s_total += 1LL << depth[t];
    max_depth = std::max(max_depth, depth[t]);
    nmax = std::max(nmax, n);
  }
  // Shared memory of the top kernel: the root and its L rows, then, when its
  // CTAs go on breadth first (emid > 0), two level buffers and per-node
  // scratch; emid shrinks until that fits in 200 KB.
  const int mid_off = sym(2 * nmax) + 4 * nmax;
  int capA_top = 1, capB_top = 1, ncap = 1;
  size_t smem_top = (size_t)mid_off * sizeof(E);
  for (int ecap = 8; ecap >= 0; --ecap) {
    int emax = 0;
    capA_top = capB_top = 1;
    for (int t = 0; t < ntrees; ++t) {
      const int e = std::min(emid[t], ecap);
      emax = std::max(emax, e);
      for (int j = 0; j <= e && e > 0; ++j) {
        const int c = (1 << j) * sym(2 * (trees[t].n - dtop[t] - j));
        if (j & 1) capB_top = std::max(capB_top, c); else capA_top = std::max(capA_top, c);
      }
    }
    ncap = 1 << emax;
    smem_top = emax == 0 ? (size_t)mid_off * sizeof(E)
                         : (size_t)(mid_off + capA_top + capB_top + ncap) * sizeof(E) +
                               (size_t)ncap * (2 * sizeof(S) + 2 * sizeof(T));
    if (smem_top <= 200 * 1024 || ecap == 0) {
      for (int t = 0; t < ntrees; ++t) emid[t] = std::min(emid[t], ecap);
      break;
    }
  }
  std::vector<TopSeg> top(ntrees);
  long long top_blocks = 0;
  for (int t = 0; t < ntrees; ++t) {
    top[t] = TopSeg{top_blocks, trees[t].root_off, region[t], sreg[t], trees[t].n, dtop[t], t,
                    (dtop[t] + emid[t]) & 1, emid[t], 0};
    top_blocks += 1LL << dtop[t];
  }
  std::vector<std::vector<LevelSeg>> levels(max_depth);
  std::vector<long long> level_threads(max_depth, 0);
  for (int l = 0; l < max_depth; ++l) {
    for (int t = 0; t < ntrees; ++t) {
      if (l < dtop[t] + emid[t] || l >= depth[t]) continue;
      const long long count = 1LL << l;
      const int q = trees[t].n - l;
      const int rows = 2 * q - 2;
      const long long g = (tune.level_threads + count - 1) / count;
      const int groups = (int)std::max(1LL, std::min<long long>(rows, g));
      levels[l].push_back(LevelSeg{level_threads[l], count, region[t], region[t], sreg[t], sreg[t], q,
                                   (rows + groups - 1) / groups, groups, t});
      level_threads[l] += count * groups;
    }
  }
  // leaf (sub_e == 0) or subtree segments, grouped by Q (one launch per distinct Q)
  // subtree CTAs have 2^sub_e threads, at least one warp; a CTA expands K = nthr / 2^el
  // consecutive roots of one tree together (el: the levels its roots expand)
  const int nthr = sub_e > 0 ? (1 << std::max(sub_e, 5)) : 128;
  std::vector<std::vector<LeafSeg>> leaf(QMAX + 1);
  std::vector<std::vector<SubSeg>> subs(QMAX + 1);
  std::vector<long long> grp_blocks(QMAX + 1, 0);
  std::vector<PartRange> ranges(ntrees);
  int capA = 1, capB = 1;
  for (int qv = QMAX; qv >= 1; --qv) {
    for (int t = 0; t < ntrees; ++t) {
      if (Q[t] != qv) continue;
      const long long count = 1LL << depth[t];
      if (sub_e > 0) {
        const int el = qroot[t] - Q[t];
        const int K = nthr >> el;
        const long long nb = (count + K - 1) / K;
        subs[qv].push_back(SubSeg{grp_blocks[qv], count, region[t], sreg[t], qroot[t], el, trees[t].n - Q[t], t,
                                  depth[t] & 1, K});
        for (int j = 0; j <= el; ++j) {
          const int c = K * (1 << j) * sym(2 * (qroot[t] - j));
          if (j & 1) capB = std::max(capB, c); else capA = std::max(capA, c);
        }
        ranges[t] = PartRange{grp_blocks[qv], nb};
        grp_blocks[qv] += nb;
      } else {
        const long long nb = (count + 127) / 128;
        leaf[qv].push_back(LeafSeg{grp_blocks[qv], count, region[t], sreg[t], depth[t], t, depth[t] & 1, 0});
        ranges[t] = PartRange{grp_blocks[qv], nb};
        grp_blocks[qv] += nb;
      }
    }
  }
  std::vector<long long> part_base(QMAX + 2, 0);
  long long parts_total = 0;
  for (int qv = QMAX; qv >= 1; --qv) {
    part_base[qv] = parts_total;
    parts_total += grp_blocks[qv];
  }
  for (int t = 0; t < ntrees; ++t) ranges[t].first += part_base[Q[t]];
  // two-stage reduction: chunks of <= 128 partials of one tree, then one warp per tree
  std::vector<PartChunk> chunks;
  std::vector<PartRange> ranges2(ntrees);
  for (int t = 0; t < ntrees; ++t) {
    ranges2[t].first = (long long)chunks.size();
    for (long long i = 0; i < ranges[t].count; i += 128)
      chunks.push_back(PartChunk{ranges[t].first + i, std::min<long long>(128, ranges[t].count - i)});
    ranges2[t].count = (long long)chunks.size() - ranges2[t].first;
  }

  // ---------------- memory
  const size_t need = 2 * (size_t)region_total * sizeof(E) + 2 * (size_t)s_total * sizeof(S) +
                      (size_t)(parts_total + chunks.size()) * sizeof(Partial<Red>);
  if (ntrees > 1 && ctx->batch_cap_bytes && need > ctx->batch_cap_bytes) {
    ctx->batch_split = true;  // the caller evaluates the batch in parts
    return GBS_ENOMEM;
  }
  gbs_status st;
  if ((st = dev_reserve(ctx, ctx->lvl[0], (size_t)region_total * sizeof(E))) ||
      (st = dev_reserve(ctx, ctx->lvl[1], (size_t)region_total * sizeof(E))) ||
      (st = dev_reserve(ctx, ctx->sbuf[0], (size_t)s_total * sizeof(S))) ||
      (st = dev_reserve(ctx, ctx->sbuf[1], (size_t)s_total * sizeof(S))) ||
      (st = dev_reserve(ctx, ctx->partials, (size_t)(parts_total + chunks.size()) * sizeof(Partial<Red>))))
    return st;
  Blob blob;
  const size_t o_top = blob.put(top);
  std::vector<size_t> o_lvl(max_depth);
  for (int l = 0; l < max_depth; ++l) o_lvl[l] = blob.put(levels[l]);
  std::vector<size_t> o_leaf(QMAX + 1);
  for (int qv = 1; qv <= QMAX; ++qv) o_leaf[qv] = sub_e > 0 ? blob.put(subs[qv]) : blob.put(leaf[qv]);
  const size_t o_chk = blob.put(chunks);
  const size_t o_rng = blob.put(ranges2);
  const unsigned char* plan = nullptr;
  if ((st = stage(ctx, blob.bytes.data(), blob.bytes.size(), (const void**)&plan))) return st;

  cudaStream_t s = ctx->stream;
  E* buf[2] = {(E*)ctx->lvl[0].ptr, (E*)ctx->lvl[1].ptr};
  S* sb[2] = {(S*)ctx->sbuf[0].ptr, (S*)ctx->sbuf[1].ptr};
  Partial<Red>* parts = (Partial<Red>*)ctx->partials.ptr;
  Partial<Red>* parts2 = parts + parts_total;

  // ---------------- top
  // The opt-in limit is set whatever the size: the kernels' static shared
  // memory (reduction scratch) counts against the default 48 KB as well.
  if ((st = check_cuda(ctx, cudaFuncSetAttribute(batch_top_kernel<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem_top),
                       "top smem")))
    return st;
  batch_top_kernel<E><<<(unsigned)top_blocks, tune.top_threads, smem_top, s>>>(
      (const TopSeg*)(plan + o_top), ntrees, (const typename root_src<E>::type*)roots_dev, buf[0], buf[1], sb[0], sb[1],
      status_dev, capA_top, capB_top, mid_off, ncap);
  count_launch(ctx);
  // ---------------- breadth-first levels
  for (int l = 0; l < max_depth; ++l) {
    if (levels[l].empty()) continue;
    const long long nt = level_threads[l];
    batch_level_kernel<E><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(
        (const LevelSeg*)(plan + o_lvl[l]), (int)levels[l].size(), nt, buf[l & 1], sb[l & 1], buf[(l + 1) & 1],
        sb[(l + 1) & 1], status_dev);
    count_launch(ctx);
  }
  // ---------------- leaves / subtrees
  if (ctx->timing) {
    if (!ctx->leaf_timer.start) {
      cudaEventCreate(&ctx->leaf_timer.start);
      cudaEventCreate(&ctx->leaf_timer.stop);
    }
    cudaEventRecord(ctx->leaf_timer.start, s);
  }
  const size_t smem_sub = (size_t)(capA + capB + nthr) * sizeof(E) + (size_t)nthr * (2 * sizeof(S) + 2 * sizeof(T));
  for (int qv = QMAX; qv >= 1; --qv) {
    const long long nb = grp_blocks[qv];
    if (nb == 0) continue;
    long long grid = nb;
    if (tune.leaf_grid_per_sm > 0) grid = std::min<long long>(nb, (long long)ctx->sm_count * tune.leaf_grid_per_sm);
    const int ns = sub_e > 0 ? (int)subs[qv].size() : (int)leaf[qv].size();
    Partial<Red>* pp = parts + part_base[qv];
    switch (qv) {
#define GBS_LEAF_CASE(QQ)                                                                                              \
  case QQ:                                                                                                             \
    if constexpr (QQ <= QMAX) {                                                                                        \
      if (sub_e > 0) {                                                                                                 \
        if ((st = check_cuda(ctx,                                                                                      \
                             cudaFuncSetAttribute(batch_subtree_kernel<E, QQ, PAIR>,                                   \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sub),         \
                             "subtree smem")))                                                                         \
          return st;                                                                                                   \
        batch_subtree_kernel<E, QQ, PAIR><<<(unsigned)grid, nthr, smem_sub, s>>>(                                      \
            (const SubSeg*)(plan + o_leaf[qv]), ns, nb, buf[0], buf[1], sb[0], sb[1], capA, capB, pp,                  \
            status_dev);                                                                                               \
      } else {                                                                                                         \
        batch_leaf_kernel<E, QQ, PAIR><<<(unsigned)grid, 128, 0, s>>>((const LeafSeg*)(plan + o_leaf[qv]), ns, nb,     \
                                                                buf[0], buf[1], sb[0], sb[1], pp, status_dev);         \
      }                                                                                                                \
    }                                                                                                                  \
    break;
      GBS_LEAF_CASE(1)
      GBS_LEAF_CASE(2)
      GBS_LEAF_CASE(3)
      GBS_LEAF_CASE(4)
      GBS_LEAF_CASE(5)
      GBS_LEAF_CASE(6)
#undef GBS_LEAF_CASE
    }
    count_launch(ctx);
  }
  if (ctx->timing) {
    cudaEventRecord(ctx->leaf_timer.stop, s);
    ctx->leaf_timer.pending = true;
  }
  // ---------------- per-tree reduction in two fixed-order stages
  batch_chunk_kernel<Red><<<(unsigned)chunks.size(), 128, 0, s>>>(parts, (const PartChunk*)(plan + o_chk),
                                                                 (int)chunks.size(), parts2);
  batch_final_kernel<Red><<<(ntrees * 32 + 255) / 256, 256, 0, s>>>(parts2, (const PartRange*)(plan + o_rng), ntrees,
                                                                     outs_dev);
  count_launch(ctx, 2);
  return check_cuda(ctx, cudaGetLastError(), "batch launch");
}

}  // namespace gbs
