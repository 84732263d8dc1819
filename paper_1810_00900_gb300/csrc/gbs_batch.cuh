// Batched subset-determinant trees: many trees of uneven size in one pass.
//
// The decision tree of gbs_tree.cuh, organised for a batch of T trees (one per
// probability request or sampler trajectory) with n_t modes each:
//
//   top kernel     one CTA per node at depth dtop_t <= D_TOP of every tree.  The
//                  CTA loads the tree's root into shared memory and eliminates
//                  its own included prefix modes in place (rank-2 Schur steps),
//                  then writes its node.  Replaces the latency-bound launches
//                  of the first levels, where nodes are few and matrices big.
//   level kernel   one launch per remaining breadth-first level, all trees that
//                  still have that level together; one thread per (node, group
//                  of rows) with the rows per thread chosen per level so that
//                  deep levels (many small nodes) do one pivot per node.
//   leaf kernel    register depth-first subtrees of the last Q levels (as in
//                  gbs_tree.cuh); blocks never straddle two trees, so each
//                  block partial belongs to one tree; optionally persistent.
//   final kernel   one warp per tree sums its block partials in a fixed order,
//                  so a tree's result does not depend on the rest of the batch.
//
// Each tree owns a fixed region of both level buffers (sized for its largest
// level), so trees at different depths never overwrite each other.
#pragma once
#include "gbs_tree_driver.cuh"

namespace gbs {

struct TopSeg {
  long long block_begin;  // first CTA of this tree
  long long root_off;     // first packed root entry of the tree
  long long out_base;     // entry offset of its output nodes (SoA, count = 2^(dtop + emid))
  long long s_base;       // offset of their s values
  int n, dtop, tree, buf;  // buf: level buffer (0/1) receiving the nodes
  int emid, pad;           // levels each CTA then expands in shared memory before writing
};

struct LevelSeg {
  long long thread_begin;
  long long count;  // parents in this segment
  long long in_base, out_base, s_in, s_out;
  int q, rpt, groups, tree;
};

struct LeafSeg {
  long long block_begin;
  long long count;  // nodes of this tree at its leaf level
  long long base, s_base;
  int depth, tree, buf, pad;
};

struct PartRange {
  long long first, count;  // block partials of one tree
};

template <class Seg, class Key>
__device__ __forceinline__ int find_seg(const Seg* segs, int nseg, Key key, Key Seg::*field) {
  int lo = 0, hi = nseg - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].*field <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Node buffers in global memory hold packed lower triangles entry-major: entry
// e of node i of a region of `count` nodes is element e * count + i.  Multiword
// entries (node_words > 0) are stored limb-major inside that: limb k of entry e
// of node i is 32-bit word (e * L + k) * count + i of the region, so every limb
// load or store of a warp covers one contiguous 128-byte line.
template <class E>
__device__ __forceinline__ E ld_node(const E* base, long long e, long long count, long long i) {
  constexpr int L = node_words<E>::value;
  if constexpr (L == 0) {
    return base[e * count + i];
  } else {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(base);
    E r;
#pragma unroll
    for (int k = 0; k < L; ++k) r.w[k] = w[(e * L + k) * count + i];
    return r;
  }
}
template <class E>
__device__ __forceinline__ void st_node(E* base, long long e, long long count, long long i, const E& v) {
  constexpr int L = node_words<E>::value;
  if constexpr (L == 0) {
    base[e * count + i] = v;
  } else {
    uint32_t* w = reinterpret_cast<uint32_t*>(base);
#pragma unroll
    for (int k = 0; k < L; ++k) w[(e * L + k) * count + i] = v.w[k];
  }
}

// packed index -> (row, col), col <= row
__device__ __forceinline__ void untri(int e, int& a, int& b) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > e) --r;
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  a = r;
  b = e - r * (r + 1) / 2;
}

// Breadth-first expansion of `levels` tree levels inside one CTA: src holds
// `nodes` nodes with q undecided modes (entry-major: entry e of node t at
// src[e * nodes + t]) and ssrc their s.  Each level replaces node t by its
// exclude child 2t and include child 2t + 1; on return src/ssrc point at the
// last level and nodes/q describe it.  Scratch: pm10, pq00, pq11 hold one
// value per node of the level being split.
template <class E>
__device__ __forceinline__ void smem_expand(E*& src, E*& dst, typename scale_of<E>::type*& ssrc,
                                            typename scale_of<E>::type*& sdst, E* pm10,
                                            typename real_of<E>::type* pq00, typename real_of<E>::type* pq11,
                                            int& nodes, int& q, int levels,
                                            bool& bad) {
  typedef typename real_of<E>::type T;
  typedef typename scale_of<E>::type S;
  const int nthr = blockDim.x;
  for (int lvl = 0; lvl < levels; ++lvl) {
    for (int t = threadIdx.x; t < nodes; t += nthr) {
      const T p00 = re_of(src[tri(0, 0) * nodes + t]);
      const T p11 = re_of(src[tri(1, 1) * nodes + t]);
      const E p10 = src[tri(1, 0) * nodes + t];
      const T det = p00 * p11 - norm2(p10);
      bad |= !is_pos(det) || !lead_pos(p00);
      const T g = rsqrt_(det);
      const T inv = g * g;
      pq00[t] = p00 * inv;
      pq11[t] = p11 * inv;
      pm10[t] = neg_(scale_(p10, inv));
      sdst[2 * t] = ssrc[t];
      sdst[2 * t + 1] = ssrc[t] * g;
    }
    __syncthreads();
    const int rows = 2 * q - 2;
    const int n2 = 2 * nodes;
    for (int task = threadIdx.x; task < nodes * rows; task += nthr) {
      const int t = task % nodes, a = task / nodes;
#define SRC(i, j) src[tri(i, j) * nodes + t]
      const E u0 = SRC(a + 2, 0), u1 = SRC(a + 2, 1);
      const E m10 = pm10[t];
      const E L0 = lin2(u0, pq11[t], u1, m10);
      const E L1 = lin2(u1, pq00[t], u0, conj_(m10));
      for (int b = 0; b < a; ++b) {
        const E x = SRC(a + 2, b + 2);
        dst[tri(a, b) * n2 + 2 * t] = x;
        dst[tri(a, b) * n2 + 2 * t + 1] = fms_conj(fms_conj(x, L0, SRC(b + 2, 0)), L1, SRC(b + 2, 1));
      }
      const E x = SRC(a + 2, a + 2);
      dst[tri(a, a) * n2 + 2 * t] = x;
      dst[tri(a, a) * n2 + 2 * t + 1] = fms_conj_re(fms_conj_re(x, L0, u0), L1, u1);
#undef SRC
    }
    __syncthreads();
    E* tmp = src; src = dst; dst = tmp;
    S* ts = ssrc; ssrc = sdst; sdst = ts;
    nodes = n2;
    --q;
  }
}

// ---------------------------------------------------------------- top ----
template <class E>
__global__ void batch_top_kernel(const TopSeg* __restrict__ segs, int nseg,
                                 const typename root_src<E>::type* __restrict__ roots, E* __restrict__ buf0,
                                 E* __restrict__ buf1, typename scale_of<E>::type* __restrict__ s0,
                                 typename scale_of<E>::type* __restrict__ s1, int* __restrict__ status, int capA,
                                 int capB, int mid_off, int ncap) {
  typedef typename real_of<E>::type T;
  typedef typename scale_of<E>::type S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* C = reinterpret_cast<E*>(smem_raw);
  const TopSeg sg = segs[find_seg(segs, nseg, (long long)blockIdx.x, &TopSeg::block_begin)];
  const long long node = (long long)blockIdx.x - sg.block_begin;
  const int d = 2 * sg.n;
  for (int i = threadIdx.x; i < sym(d); i += blockDim.x) C[i] = conv_entry<E>(roots[sg.root_off + i]);
  __syncthreads();
  E* Lrow = C + sym(d);  // L0 of row a at Lrow[2a], L1 at Lrow[2a+1]
  S s = from_double<S>(1.0);
  bool bad = false;
  for (int i = 0; i < sg.dtop; ++i) {
    if (!((node >> (sg.dtop - 1 - i)) & 1)) continue;  // excluded: the view just moves on
    const int o = 2 * i;
    const T p00 = re_of(C[tri(o, o)]), p11 = re_of(C[tri(o + 1, o + 1)]);
    const E p10 = C[tri(o + 1, o)];
    const T det = p00 * p11 - norm2(p10);
    bad |= !is_pos(det) || !lead_pos(p00);
    const T g = rsqrt_(det);
    const T inv = g * g;
    const T q00 = p00 * inv, q11 = p11 * inv;
    const E m10 = neg_(scale_(p10, inv));
    s = s * g;
    for (int a = o + 2 + threadIdx.x; a < d; a += blockDim.x) {
      const E ua0 = C[tri(a, o)], ua1 = C[tri(a, o + 1)];
      Lrow[2 * a] = lin2(ua0, q11, ua1, m10);
      Lrow[2 * a + 1] = lin2(ua1, q00, ua0, conj_(m10));
    }
    __syncthreads();
    const int rest = d - o - 2;  // trailing block rows
    for (int e = threadIdx.x; e < sym(rest); e += blockDim.x) {
      int a, b;
      untri(e, a, b);
      a += o + 2;
      b += o + 2;
      const E L0 = Lrow[2 * a], L1 = Lrow[2 * a + 1];
      if (a == b) {
        C[tri(a, a)] = fms_conj_re(fms_conj_re(C[tri(a, a)], L0, C[tri(a, o)]), L1, C[tri(a, o + 1)]);
      } else {
        C[tri(a, b)] = fms_conj(fms_conj(C[tri(a, b)], L0, C[tri(b, o)]), L1, C[tri(b, o + 1)]);
      }
    }
    __syncthreads();
  }
  const int o = 2 * sg.dtop;
  const int dq = d - o;
  E* out = sg.buf ? buf1 : buf0;
  S* sout = sg.buf ? s1 : s0;
  if (sg.emid == 0) {
    const long long cnt = 1LL << sg.dtop;
    for (int e = threadIdx.x; e < sym(dq); e += blockDim.x) {
      int a, b;
      untri(e, a, b);
      st_node(out + sg.out_base, e, cnt, node, C[tri(a + o, b + o)]);
    }
    if (threadIdx.x == 0) sout[sg.s_base + node] = s;
  } else {
    // The node goes on breadth first in shared memory for emid more levels and
    // writes its 2^emid descendants (node index (node << emid) | t at that depth).
    E* src = reinterpret_cast<E*>(smem_raw) + mid_off;
    E* dst = src + capA;
    E* pm10 = dst + capB;
    S* ssrc = reinterpret_cast<S*>(pm10 + ncap);
    S* sdst = ssrc + ncap;
    T* pq00 = reinterpret_cast<T*>(sdst + ncap);
    T* pq11 = pq00 + ncap;
    for (int e = threadIdx.x; e < sym(dq); e += blockDim.x) {
      int a, b;
      untri(e, a, b);
      src[e] = C[tri(a + o, b + o)];
    }
    if (threadIdx.x == 0) ssrc[0] = s;
    __syncthreads();
    int nodes = 1, q = sg.n - sg.dtop;
    smem_expand<E>(src, dst, ssrc, sdst, pm10, pq00, pq11, nodes, q, sg.emid, bad);
    const long long cnt = 1LL << (sg.dtop + sg.emid);
    const long long first = node << sg.emid;
    for (int i = threadIdx.x; i < sym(2 * q) * nodes; i += blockDim.x) {
      const int e = i / nodes, t = i - e * nodes;
      st_node(out + sg.out_base, e, cnt, first + t, src[i]);
    }
    for (int t = threadIdx.x; t < nodes; t += blockDim.x) sout[sg.s_base + first + t] = ssrc[t];
  }
  if (bad) atomicExch(status + sg.tree, bad_status<typename real_of<E>::type>());
}

// ---------------------------------------------------------------- level --
template <class E>
__global__ void __launch_bounds__(256, level_min_blocks<E>::value) batch_level_kernel(const LevelSeg* __restrict__ segs, int nseg, long long total,
                                   const E* __restrict__ in, const typename scale_of<E>::type* __restrict__ sin,
                                   E* __restrict__ out, typename scale_of<E>::type* __restrict__ sout,
                                   int* __restrict__ status) {
  typedef typename real_of<E>::type T;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= total) return;
  const LevelSeg sg = segs[find_seg(segs, nseg, tid, &LevelSeg::thread_begin)];
  const long long local = tid - sg.thread_begin;
  const long long count = sg.count;
  // With up to 8 row groups, threads go over tiles of 32 consecutive nodes (the
  // whole level when it has fewer): a warp holds one row group of 32 nodes and a
  // 256-thread CTA whole tiles, so the parent entries all groups read (pivot
  // block, first two columns) are still cached when the later groups read them,
  // and a CTA's warps carry every row group (equal work).  With more groups a CTA
  // would hold a few row groups of unequal cost; there one row group of
  // consecutive nodes per CTA keeps its warps' work equal.
  long long node;
  int grp;
  if (sg.groups <= 8) {
    const long long tile = (count & 31) ? count : 32;
    const long long within = local % (tile * sg.groups);
    node = (local / (tile * sg.groups)) * tile + within % tile;
    grp = (int)(within / tile);
  } else {
    node = local % count;
    grp = (int)(local / count);
  }
  const int rows = 2 * sg.q - 2;
  const E* par = in + sg.in_base;
  const long long c2 = 2 * count;
  E* chi = out + sg.out_base;
#define PAR(i, j) ld_node(par, tri(i, j), count, node)
  const T p00 = re_of(PAR(0, 0));
  const T p11 = re_of(PAR(1, 1));
  const E p10 = PAR(1, 0);
  const T det = p00 * p11 - norm2(p10);
  if (!is_pos(det) || !lead_pos(p00)) {
    if (grp == 0) atomicExch(status + sg.tree, bad_status<typename real_of<E>::type>());
    return;
  }
  const T g = rsqrt_(det);
  const T inv = g * g;
  const T q00 = p00 * inv, q11 = p11 * inv;
  const E m10 = neg_(scale_(p10, inv));
  // Fixed-point entries (level_park): the scaled pivot inverse and g wait in this
  // thread's shared-memory slot while the rows are formed (read back once per
  // row), which frees the registers the row loop would otherwise spill.
  constexpr int LW = node_words<E>::value;
  constexpr bool PARK = level_park<E>::value && LW > 0;
  __shared__ uint32_t park[PARK ? 4 * LW : 1][PARK ? 256 : 1];
  if constexpr (PARK) {
#pragma unroll
    for (int k = 0; k < LW; ++k) {
      park[k][threadIdx.x] = q00.w[k];
      park[LW + k][threadIdx.x] = q11.w[k];
      park[2 * LW + k][threadIdx.x] = m10.w[k];
      park[3 * LW + k][threadIdx.x] = g.w[k];
    }
  }
  auto unpark = [&](int slot, const auto& keep) {
    typedef typename std::decay<decltype(keep)>::type V;
    if constexpr (PARK) {
      V r;
      const volatile uint32_t* src = &park[slot * LW][threadIdx.x];
#pragma unroll
      for (int k = 0; k < LW; ++k) r.w[k] = src[k * 256];
      return r;
    } else {
      return keep;
    }
  };
  for (int a = grp; a < rows; a += sg.groups) {
    const E u0 = PAR(a + 2, 0), u1 = PAR(a + 2, 1);
    const E m10r = unpark(2, m10);
    const E L0 = lin2(u0, unpark(1, q11), u1, m10r);
    const E L1 = lin2(u1, unpark(0, q00), u0, conj_(m10r));
    for (int b = 0; b < a; ++b) {
      const E x = PAR(a + 2, b + 2);
      E v = fms_conj(x, L0, PAR(b + 2, 0));
      v = fms_conj(v, L1, PAR(b + 2, 1));
      st_node(chi, tri(a, b), c2, 2 * node, x);
      st_node(chi, tri(a, b), c2, 2 * node + 1, v);
    }
    const E x = PAR(a + 2, a + 2);
    E v = fms_conj_re(x, L0, u0);
    v = fms_conj_re(v, L1, u1);
    st_node(chi, tri(a, a), c2, 2 * node, x);
    st_node(chi, tri(a, a), c2, 2 * node + 1, v);
  }
  if (grp == 0) {
    const typename scale_of<E>::type s = sin[sg.s_in + node];
    sout[sg.s_out + 2 * node] = s;
    sout[sg.s_out + 2 * node + 1] = s * unpark(3, g);
  }
#undef PAR
}

// ----------------------------------------------------------------- leaf --
template <class E, int Q, bool PAIR = false>
__global__ void __launch_bounds__(128, leaf_min_blocks<E>::value) batch_leaf_kernel(const LeafSeg* __restrict__ segs, int nseg,
                                                         long long total_blocks, const E* __restrict__ buf0,
                                                         const E* __restrict__ buf1,
                                                         const typename scale_of<E>::type* __restrict__ s0,
                                                         const typename scale_of<E>::type* __restrict__ s1,
                                                         Partial<typename acc_traits<typename real_of<E>::type>::Red>* parts,
                                                         int* __restrict__ status) {
  typedef typename real_of<E>::type T;
  typedef typename acc_traits<T>::Acc Acc;
  typedef typename acc_traits<T>::Red Red;
  for (long long vb = blockIdx.x; vb < total_blocks; vb += gridDim.x) {
    const LeafSeg sg = segs[find_seg(segs, nseg, vb, &LeafSeg::block_begin)];
    const long long node = (vb - sg.block_begin) * blockDim.x + threadIdx.x;
    if constexpr (std::is_same<Acc, double>::value) {
      Sums<double> a = sums_zero<double>();
      if (node < sg.count) {
        const E* nodes = (sg.buf ? buf1 : buf0) + sg.base;
        E c[sym(2 * Q)];
#pragma unroll
        for (int e = 0; e < sym(2 * Q); ++e) c[e] = ld_node(nodes, e, sg.count, node);
        const typename scale_of<E>::type s = (sg.buf ? s1 : s0)[sg.s_base + node];
        const bool ok = subtree_run<E, Q, PAIR>(c, s, a);
        if (!ok || !isfinite((a.ip + a.in) + (a.ep + a.en))) atomicExch(status + sg.tree, bad_status<T>());
        if ((sg.depth - __popcll((unsigned long long)node)) & 1) {
          const double t0 = a.ip, t1 = a.ep;
          a.ip = a.in; a.in = t0; a.ep = a.en; a.en = t1;
        }
      }
      block_reduce_sums<PAIR>(a.ip, a.in, a.ep, a.en, parts + vb);
    } else {
      Red inc = red_zero<Red>(), exc = red_zero<Red>();
      double asum = 0.0;
      if (node < sg.count) {
        const E* nodes = (sg.buf ? buf1 : buf0) + sg.base;
        E c[sym(2 * Q)];
#pragma unroll
        for (int e = 0; e < sym(2 * Q); ++e) c[e] = ld_node(nodes, e, sg.count, node);
        const typename scale_of<E>::type s = (sg.buf ? s1 : s0)[sg.s_base + node];
        if (!subtree_sums<E, Q, PAIR>(c, s, inc, exc, asum)) atomicExch(status + sg.tree, bad_status<T>());
        if ((sg.depth - __popcll((unsigned long long)node)) & 1) {
          inc = red_neg(inc);
          exc = red_neg(exc);
        }
      }
      block_reduce_store(inc, exc, asum, parts + vb);
    }
    __syncthreads();
  }
}

// -------------------------------------------------------------- subtree --
// One CTA per k_roots consecutive nodes with q_root undecided modes (of one
// tree): breadth-first expansion of the first e_levels levels of all of them
// together in shared memory (two ping-pong level buffers, node matrices
// entry-major), then one thread per resulting node runs the register
// depth-first subtree of the last Q levels.  One partial per CTA.
struct SubSeg {
  long long block_begin;  // first CTA of this tree
  long long count;        // subtree roots of this tree
  long long base, s_base; // where the roots are (level buffer `buf`)
  int q_root, e_levels, depth_leaf, tree, buf, k_roots;
};

template <class E, int Q, bool PAIR = false>
__global__ void __launch_bounds__(128) batch_subtree_kernel(
    const SubSeg* __restrict__ segs, int nseg, long long total_blocks, const E* __restrict__ buf0,
    const E* __restrict__ buf1, const typename scale_of<E>::type* __restrict__ s0,
    const typename scale_of<E>::type* __restrict__ s1, int capA, int capB,
    Partial<typename acc_traits<typename real_of<E>::type>::Red>* parts, int* __restrict__ status) {
  typedef typename real_of<E>::type T;
  typedef typename acc_traits<T>::Acc Acc;
  typedef typename acc_traits<T>::Red Red;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nthr = blockDim.x;
  E* bufA = reinterpret_cast<E*>(smem_raw);
  E* bufB = bufA + capA;
  E* pm10 = bufB + capB;                           // per node of the current level
  typedef typename scale_of<E>::type S;
  S* sA = reinterpret_cast<S*>(pm10 + nthr);       // s of the current level
  S* sB = sA + nthr;
  T* pq00 = reinterpret_cast<T*>(sB + nthr);
  T* pq11 = pq00 + nthr;
  for (long long vb = blockIdx.x; vb < total_blocks; vb += gridDim.x) {
    const SubSeg sg = segs[find_seg(segs, nseg, vb, &SubSeg::block_begin)];
    const long long root = (vb - sg.block_begin) * sg.k_roots;  // first root of this CTA
    const int nroots = (int)min((long long)sg.k_roots, sg.count - root);
    const E* rsrc = (sg.buf ? buf1 : buf0) + sg.base;
    int q = sg.q_root;
    for (int i = threadIdx.x; i < sym(2 * q) * nroots; i += nthr) {
      const int e = i / nroots, k = i - e * nroots;
      bufA[i] = ld_node(rsrc, e, sg.count, root + k);
    }
    for (int k = threadIdx.x; k < nroots; k += nthr) sA[k] = (sg.buf ? s1 : s0)[sg.s_base + root + k];
    __syncthreads();
    E* src = bufA;
    E* dst = bufB;
    S* ssrc = sA;
    S* sdst = sB;
    int nodes = nroots;
    bool bad = false;
    smem_expand<E>(src, dst, ssrc, sdst, pm10, pq00, pq11, nodes, q, sg.e_levels, bad);
    if (bad) atomicExch(status + sg.tree, bad_status<typename real_of<E>::type>());
    const int t = threadIdx.x;
    if constexpr (std::is_same<Acc, double>::value) {
      Sums<double> a = sums_zero<double>();
      if (t < nodes) {
        E c[sym(2 * Q)];
#pragma unroll
        for (int e = 0; e < sym(2 * Q); ++e) c[e] = src[e * nodes + t];
        const bool ok = subtree_run<E, Q, PAIR>(c, ssrc[t], a);
        if (!ok || !isfinite((a.ip + a.in) + (a.ep + a.en))) atomicExch(status + sg.tree, bad_status<T>());
        const unsigned long long gnode = ((unsigned long long)root << sg.e_levels) + (unsigned long long)t;
        if ((sg.depth_leaf - __popcll(gnode)) & 1) {
          const double t0 = a.ip, t1 = a.ep;
          a.ip = a.in; a.in = t0; a.ep = a.en; a.en = t1;
        }
      }
      block_reduce_sums<PAIR>(a.ip, a.in, a.ep, a.en, parts + vb);
    } else {
      Red inc = red_zero<Red>(), exc = red_zero<Red>();
      double asum = 0.0;
      if (t < nodes) {
        E c[sym(2 * Q)];
#pragma unroll
        for (int e = 0; e < sym(2 * Q); ++e) c[e] = src[e * nodes + t];
        const S sv = ssrc[t];
        if (!subtree_sums<E, Q, PAIR>(c, sv, inc, exc, asum)) atomicExch(status + sg.tree, bad_status<T>());
        const unsigned long long gnode = ((unsigned long long)root << sg.e_levels) + (unsigned long long)t;
        if ((sg.depth_leaf - __popcll(gnode)) & 1) {
          inc = red_neg(inc);
          exc = red_neg(exc);
        }
      }
      block_reduce_store(inc, exc, asum, parts + vb);
    }
    __syncthreads();
  }
}

// Stage one of the per-tree reduction: chunk c sums partials [first, first+count)
// of one tree in order.
struct PartChunk {
  long long first, count;
};

template <class Red>
__global__ void batch_chunk_kernel(const Partial<Red>* __restrict__ parts, const PartChunk* __restrict__ chunks,
                                   int nchunks, Partial<Red>* __restrict__ out) {
  const int c = blockIdx.x;
  if (c >= nchunks) return;
  const PartChunk ch = chunks[c];
  Red inc = red_zero<Red>(), exc = red_zero<Red>();
  double asum = 0.0;
  if (threadIdx.x < ch.count) {
    inc = parts[ch.first + threadIdx.x].inc;
    exc = parts[ch.first + threadIdx.x].exc;
    asum = parts[ch.first + threadIdx.x].abs;
  }
  block_reduce_store(inc, exc, asum, out + c);
}

// ---------------------------------------------------------------- final --
template <class Red>
__global__ void batch_final_kernel(const Partial<Red>* __restrict__ parts, const PartRange* __restrict__ ranges,
                                   int ntrees, TreeOut* __restrict__ outs) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= ntrees) return;
  const PartRange r = ranges[t];
  Red inc = red_zero<Red>(), exc = red_zero<Red>();
  double asum = 0.0;
  for (long long i = lane; i < r.count; i += 32) {
    inc = red_add(inc, parts[r.first + i].inc);
    exc = red_add(exc, parts[r.first + i].exc);
    asum += parts[r.first + i].abs;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    inc = red_add(inc, shfl_down(inc, off));
    exc = red_add(exc, shfl_down(exc, off));
    asum += __shfl_down_sync(0xffffffffu, asum, off);
  }
  if (lane == 0) {
    red_store(inc, outs[t].inc);
    red_store(exc, outs[t].exc);
    outs[t].abs = asum;
  }
}

}  // namespace gbs
