// Subset-determinant decision tree (the hot path).
//
// For a 2n x 2n Hermitian (complex basis) or symmetric (real x/p basis)
// positive-definite matrix G, whose rows 2i, 2i+1 belong to mode i, the tree
// enumerates all 2^n mode subsets Z and the terms det(G_Z)^(-1/2), summed as
//   f_inc = sum over Z containing the last mode  of (-1)^(n-|Z|) det(G_Z)^(-1/2)
//   f_exc = sum over Z without the last mode     of (-1)^(n-|Z|) det(G_Z)^(-1/2)
//   abs   = sum over all Z of det(G_Z)^(-1/2)
// With G = (Sigma^-1)_S this gives the Torontonian Tor(O_S) = f_inc + f_exc;
// with G a conditioned Sigma' over S u {k} (k last) it gives both sums of the
// chain-rule sampler's no-click probability.  Every term is one of the paper's
// vacuum probabilities (Eq. 5), and the signed sums are its click/no-click
// bookkeeping (Eqs. 6-7) in closed form.
//
// Tree: decide the modes in order.  A node with q undecided modes holds C, the
// Schur complement of those modes given the included ones, and s, the product
// of det(P)^(-1/2) over the included pivots P, so that at a leaf
// s = det(G_Z)^(-1/2) (block elimination: det [[P, B], [B^H, D]] = det P *
// det(D - B^H P^-1 B), the identity behind the paper's Eq. 4a).  Excluding the
// first undecided mode drops its two rows; including it replaces C by
// C - C[:, p] P^-1 C[p, :] (a rank-2 update) and s by s det(P)^(-1/2).
//
// Work split:
//   levels 0 .. n-Q-1   breadth first, one kernel per level, one thread per
//                       (node, row of the child); node matrices live in global
//                       memory as packed lower triangles, entry-major (SoA).
//   last Q levels       one thread per node: a depth-first subtree unrolled at
//                       compile time with every matrix in registers; all 32
//                       lanes of a warp run the identical instruction stream on
//                       different nodes (the tree is perfectly regular).
//   reduction           per-block partials in the accumulation type, then one
//                       block sums them in a fixed order (bitwise deterministic).
#pragma once
#include <type_traits>

#include "gbs_num.cuh"

namespace gbs {

constexpr int sym(int d) { return d * (d + 1) / 2; }
GBS_HD constexpr int tri(int a, int b) { return a * (a + 1) / 2 + b; }  // b <= a

template <class E, class T>
GBS_HD E scale_(const E& x, const T& s);
template <>
GBS_HD double scale_<double, double>(const double& x, const double& s) { return x * s; }
template <>
GBS_HD float scale_<float, float>(const float& x, const float& s) { return x * s; }
template <>
GBS_HD dd scale_<dd, dd>(const dd& x, const dd& s) { return x * s; }
template <>
GBS_HD td scale_<td, td>(const td& x, const td& s) { return x * s; }
template <>
GBS_HD cplx<double> scale_<cplx<double>, double>(const cplx<double>& x, const double& s) { return {x.re * s, x.im * s}; }
template <>
GBS_HD cplx<float> scale_<cplx<float>, float>(const cplx<float>& x, const float& s) { return {x.re * s, x.im * s}; }
template <>
GBS_HD cplx<dd> scale_<cplx<dd>, dd>(const cplx<dd>& x, const dd& s) { return {x.re * s, x.im * s}; }
template <>
GBS_HD cplx<td> scale_<cplx<td>, td>(const cplx<td>& x, const td& s) { return {x.re * s, x.im * s}; }

// Type of the running product s of pivot factors: the entry scalar type,
// except for the fixed-point entries, whose s needs a wider integer part.
template <class E> struct scale_of { typedef typename real_of<E>::type type; };

// Minimum resident CTAs per SM the compiler keeps registers for in the
// breadth-first level kernel: the fixed-point levels wait on global loads with
// too few warps otherwise.
template <class E> struct level_min_blocks { static const int value = 1; };
// Level kernel: keep the scaled pivot inverse and g in shared memory while the
// rows are formed (the fixed-point entry types, whose registers would otherwise
// spill).
template <class E> struct level_park { static const bool value = false; };
// The same for the register-subtree leaf kernel (128-thread CTAs).
template <class E> struct leaf_min_blocks { static const int value = 1; };

// 32-bit words of a multiword entry stored limb by limb in the global node
// buffers of the batched engine (0: the entry is stored whole).
template <class E> struct node_words { static const int value = 0; };

// ------------------------------------------------ accumulation types -----
// Per-thread accumulators (Acc) and cross-thread reduction values (Red).
template <class T> struct acc_traits;
template <> struct acc_traits<double> { typedef double Acc; typedef dd Red; };
template <> struct acc_traits<float> { typedef double Acc; typedef dd Red; };
template <> struct acc_traits<dd> { typedef dd Acc; typedef dd Red; };
template <> struct acc_traits<td> { typedef td Acc; typedef td Red; };

GBS_HD void acc_add(double& a, double x) { a += x; }
GBS_HD void acc_add(double& a, float x) { a += (double)x; }
GBS_HD void acc_add(dd& a, const dd& x) { a = a + x; }
GBS_HD void acc_add(td& a, const td& x) { a = a + x; }

// acc += a * b (the term s * g of an included leaf)
GBS_HD void acc_fpa(double& acc, double a, double b) { acc = fma(a, b, acc); }
GBS_HD void acc_fpa(double& acc, float a, float b) { acc += (double)(a * b); }
GBS_HD void acc_fpa(dd& acc, const dd& a, const dd& b) { acc = acc + a * b; }
GBS_HD void acc_fpa(td& acc, const td& a, const td& b) { acc = acc + a * b; }

// Per-thread term sums split by sign: no sum cancels inside a thread, each
// leaf pair costs two accumulations, and the absolute sum comes for free:
// f_inc = ip - in, f_exc = ep - en, abs = ip + in + ep + en.
template <class Acc>
struct Sums {
  Acc ip, in, ep, en;
};
// Sum of |terms| of a thread's sign-split sums as a double (specialised where the
// sums are exact integers: add first, convert once).
template <class Acc>
struct sums_total {
  static GBS_HD double of(const Sums<Acc>& a) {
    return to_double(a.ip) + to_double(a.in) + (to_double(a.ep) + to_double(a.en));
  }
};
template <class Acc>
GBS_HD Sums<Acc> sums_zero() {
  const Acc z = from_double<Acc>(0.0);
  return Sums<Acc>{z, z, z, z};
}

// A pivot determinant that is not positive: the floating types need no test
// on the hot path (the inverse square root of a value <= 0 is NaN or inf and
// reaches the sums, which are checked once per thread).
GBS_HD bool not_positive(double) { return false; }
GBS_HD bool not_positive(float) { return false; }
GBS_HD bool not_positive(const dd&) { return false; }
GBS_HD bool not_positive(const td&) { return false; }

GBS_HD dd red_add(const dd& a, const dd& b) { return a + b; }
GBS_HD td red_add(const td& a, const td& b) { return a + b; }
GBS_HD dd red_neg(const dd& a) { return -a; }
GBS_HD td red_neg(const td& a) { return -a; }
GBS_HD void red_store(const dd& a, double* o) { o[0] = a.hi; o[1] = a.lo; o[2] = 0.0; }
GBS_HD void red_store(const td& a, double* o) { o[0] = a.x0; o[1] = a.x1; o[2] = a.x2; }
template <class R> GBS_HD R red_zero();
template <> GBS_HD dd red_zero<dd>() { return dd_make(0.0); }
template <> GBS_HD td red_zero<td>() { return td_make(0.0); }

__device__ __forceinline__ dd shfl_down(const dd& v, int off) {
  return dd{__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}
__device__ __forceinline__ td shfl_down(const td& v, int off) {
  return td{__shfl_down_sync(0xffffffffu, v.x0, off), __shfl_down_sync(0xffffffffu, v.x1, off),
            __shfl_down_sync(0xffffffffu, v.x2, off)};
}

template <class Red>
struct Partial {
  Red inc, exc;
  double abs;
};

// Result of one tree, as plain doubles: value = x[0] + x[1] + x[2].
struct TreeOut {
  double inc[3];
  double exc[3];
  double abs;
};

// ------------------------------------------------- device status codes ---
// kStatusRange: a fixed-point tree met a value outside the range it can carry
// (the caller redoes the tree in floating point).
enum : int { kStatusOk = 0, kStatusNotPD = 3, kStatusRange = 5 };
template <class T> constexpr int bad_status() { return kStatusNotPD; }

GBS_HD bool is_pos(double x) { return x > 0.0; }
GBS_HD bool is_pos(float x) { return x > 0.0f; }
GBS_HD bool is_pos(const dd& x) { return x.hi > 0.0; }
GBS_HD bool is_pos(const td& x) { return x.x0 > 0.0; }
// The first diagonal entry of a pivot block is positive: with det > 0 the 2 x 2
// block is then positive definite (det > 0 alone admits a negative definite one).
GBS_HD bool lead_pos(double x) { return x > 0.0; }
GBS_HD bool lead_pos(float x) { return x > 0.0f; }
GBS_HD bool lead_pos(const dd& x) { return x.hi > 0.0; }
GBS_HD bool lead_pos(const td& x) { return x.x0 > 0.0; }

// --------------------------------------------------- breadth-first level --
// Parents: count nodes with q undecided modes, entry e of node i at par[e*count + i].
// Children: 2*count nodes with q-1 modes; child 2i excludes the first mode of
// node i, child 2i+1 includes it.
template <class E>
__global__ void tree_level_kernel(const E* __restrict__ par, const typename scale_of<E>::type* __restrict__ spar,
                                  long long count, int q, E* __restrict__ chi,
                                  typename scale_of<E>::type* __restrict__ schi, int* __restrict__ status) {
  typedef typename real_of<E>::type T;
  typedef typename scale_of<E>::type S;
  const int rows = 2 * q - 2;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= count * rows) return;
  const long long node = tid % count;
  const int a = (int)(tid / count);
  const long long c2 = 2 * count;
#define PAR(i, j) par[(long long)tri(i, j) * count + node]
  const T p00 = re_of(PAR(0, 0));
  const T p11 = re_of(PAR(1, 1));
  const E p10 = PAR(1, 0);
  const T det = p00 * p11 - norm2(p10);
  if (!(to_double(det) > 0.0) || !(to_double(p00) > 0.0)) {
    if (a == 0) atomicExch(status, (int)kStatusNotPD);
    return;
  }
  const T g = rsqrt_(det);
  const T inv = g * g;
  const T q00 = p00 * inv, q11 = p11 * inv;
  const E m10 = neg_(scale_(p10, inv));  // -p10 / det
  const E u0 = PAR(a + 2, 0), u1 = PAR(a + 2, 1);
  const E L0 = lin2(u0, q11, u1, m10);           // (u0 p11 - u1 p10) / det
  const E L1 = lin2(u1, q00, u0, conj_(m10));    // (u1 p00 - u0 conj(p10)) / det
  for (int b = 0; b < a; ++b) {
    const E x = PAR(a + 2, b + 2);
    E v = fms_conj(x, L0, PAR(b + 2, 0));
    v = fms_conj(v, L1, PAR(b + 2, 1));
    chi[(long long)tri(a, b) * c2 + 2 * node] = x;
    chi[(long long)tri(a, b) * c2 + 2 * node + 1] = v;
  }
  {
    const E x = PAR(a + 2, a + 2);
    E v = fms_conj_re(x, L0, u0);
    v = fms_conj_re(v, L1, u1);
    chi[(long long)tri(a, a) * c2 + 2 * node] = x;
    chi[(long long)tri(a, a) * c2 + 2 * node + 1] = v;
  }
  if (a == 0) {
    const S s = spar[node];
    schi[2 * node] = s;
    schi[2 * node + 1] = s * g;
  }
#undef PAR
}

// ------------------------------------ last two levels without cancellation --
// The four leaves below a node with two undecided modes a, b (in that order)
// carry g_a g_c, -g_a, -g_b, +1 times the node's s and sign, where g_x =
// det(P_x)^(-1/2) for the pivot blocks P_a, P_b and P_c = P_b - D of b given a
// (D = B P_a^-1 B^T, B the b-by-a block).  Their sum is rewritten as
//   v = (g_a - 1)(g_c - 1) + (g_c - g_b)
// with every factor evaluated to a small relative error:
//   g - 1 from x = det(P) - 1 = (1 - p00)(1 - p11) - p01^2 - 1 formed from the
//     deviations o = 1 - p, then one Newton step on (1 + h)^2 (1 + x) = 1
//     from h = g - 1;
//   g_c - g_b from delta = det(P_c) - det(P_b) = -tr(adj(P_b) D) + det D, then
//     one Newton step on (g_b + y)^2 (det P_b + delta) = g_b^2 det P_b from
//     y = g_c - g_b.
// The alternating sum then adds one v per four subsets, and the terms that
// cancelled inside each group never reach it.  The magnitude a group reports
// for the error estimate covers both the rounding of its two parts and the
// first-order effect of relative perturbations of its input entries:
//   m = |(g_a-1)(g_c-1)| + |g_c-g_b| + |g_a-1| g_c + |g_c-1| g_a + |D00| + |D11|
// (the pivot blocks enter v through the small factors g - 1, the coupling B
// through D), so that sum s m / |Tor| replaces sum|t| / |Tor| in the estimate
// (1e2 to 1e3 smaller on the 200-mode states).  Real basis, FP64 only.
__device__ __forceinline__ double pair_hm1(double p00, double p11, double p01, double det, double g) {
  const double o00 = 1.0 - p00, o11 = 1.0 - p11;
  const double x = fma(-p01, p01, fma(o00, o11, -(o00 + o11)));
  const double h = g - 1.0;
  const double r = fma(h * (2.0 + h), det, x);  // (1 + h)^2 det - 1
  return fma(-0.5 * g, r, h);
}

// Adds (-1)^NEG s v to acc.ip and s m to acc.ep.
template <int D, int OFF, bool NEG>
__device__ __forceinline__ void pair_group(const double (&c)[sym(D)], double s, Sums<double>& acc) {
  const double a00 = c[tri(OFF, OFF)], a11 = c[tri(OFF + 1, OFF + 1)], a01 = c[tri(OFF + 1, OFF)];
  const double b00 = c[tri(OFF + 2, OFF + 2)], b11 = c[tri(OFF + 3, OFF + 3)], b01 = c[tri(OFF + 3, OFF + 2)];
  const double u00 = c[tri(OFF + 2, OFF)], u01 = c[tri(OFF + 2, OFF + 1)];
  const double u10 = c[tri(OFF + 3, OFF)], u11 = c[tri(OFF + 3, OFF + 1)];
  const double da = fma(a00, a11, -a01 * a01);
  const double ga = rsqrt_(da);
  const double inv = ga * ga;
  const double q00 = a00 * inv, q11 = a11 * inv, m = -a01 * inv;
  // rows of B P_a^-1, then D = B P_a^-1 B^T
  const double l0 = fma(u00, q11, u01 * m), l1 = fma(u01, q00, u00 * m);
  const double k0 = fma(u10, q11, u11 * m), k1 = fma(u11, q00, u10 * m);
  const double d00 = fma(l0, u00, l1 * u01);
  const double d11 = fma(k0, u10, k1 * u11);
  const double d01 = fma(k0, u00, k1 * u01);
  const double c00 = b00 - d00, c11 = b11 - d11, c01 = b01 - d01;
  const double db = fma(b00, b11, -b01 * b01);
  const double dc = fma(c00, c11, -c01 * c01);
  const double gb = rsqrt_(db), gc = rsqrt_(dc);
  const double ha = pair_hm1(a00, a11, a01, da, ga);
  const double hc = pair_hm1(c00, c11, c01, dc, gc);
  const double delta = fma(d00, d11, -d01 * d01) - fma(b11, d00, fma(b00, d11, -2.0 * b01 * d01));
  double y = gc - gb;
  const double f = fma(gb * gb, delta, y * (2.0 * gb + y) * (db + delta));
  y = fma(-0.5 * gc, f, y);
  const double hh = ha * hc;
  const double v = hh + y;
  if (NEG) acc.ip = fma(-s, v, acc.ip); else acc.ip = fma(s, v, acc.ip);
  const double m_in = fma(fabs(ha), gc, fabs(hc) * ga) + (fabs(d00) + fabs(d11));
  acc.ep = fma(s, (fabs(hh) + fabs(y)) + m_in, acc.ep);
}

// A tree of one mode: Tor = g - 1 (magnitude |g - 1| + g: the pivot block
// enters with the full g).
template <int D, int OFF, bool NEG>
__device__ __forceinline__ void pair_single(const double (&c)[sym(D)], double s, Sums<double>& acc) {
  const double p00 = c[tri(OFF, OFF)], p11 = c[tri(OFF + 1, OFF + 1)], p01 = c[tri(OFF + 1, OFF)];
  const double det = fma(p00, p11, -p01 * p01);
  const double g = rsqrt_(det);
  const double h = pair_hm1(p00, p11, p01, det, g);
  if (NEG) acc.ip = fma(-s, h, acc.ip); else acc.ip = fma(s, h, acc.ip);
  acc.ep = fma(s, fabs(h) + g, acc.ep);
}

// ----------------------------------------------- register depth-first ----
// Node with Q undecided modes whose matrix is the view c[tri(OFF + i, OFF + j)]
// of an array of dimension D; NEG = odd number of exclusions above it.  PAIR:
// the last two levels as cancellation-free groups (above; E = double only).
template <class E, int Q, int D, int OFF, bool NEG, bool PAIR = false>
struct Dfs {
  typedef typename real_of<E>::type T;
  typedef typename acc_traits<T>::Acc Acc;
  typedef typename scale_of<E>::type S;
  static __device__ __forceinline__ void run(const E (&c)[sym(D)], const S& s, Sums<Acc>& acc, bool& bad) {
    if constexpr (PAIR && Q <= 2) {
      static_assert(std::is_same<E, double>::value, "the paired last levels are FP64 real-basis only");
      if constexpr (Q == 2) pair_group<D, OFF, NEG>(c, s, acc); else pair_single<D, OFF, NEG>(c, s, acc);
    } else if constexpr (std::is_same<E, double>::value) {
      // FP64 real basis, the pivot block factored as P = R R^T (Cholesky):
      //   r0 = p00^(-1/2), w = p10 r0, d1 = p11 - w^2, r1 = d1^(-1/2),
      //   det(P)^(-1/2) = r0 r1,
      // and the rank-2 update as C' = C - W W^T with the rows of W = U R^-T:
      //   w0 = u0 r0,  w1 = (u1 - w0 w) r1 = u1 r1 + u0 (-w r0 r1),
      // three FP64 instructions per row where u P^-1 takes four; an entry still
      // costs two fused multiply-adds.  A one-mode node needs only det(P).
      const double p00 = c[tri(OFF, OFF)], p11 = c[tri(OFF + 1, OFF + 1)], p10 = c[tri(OFF + 1, OFF)];
      if constexpr (Q == 1) {
        // det > 0 alone admits a negative definite block: p00 > 0 is tested on its bits
        // (integer pipe), and a failed test turns g into NaN like any other bad pivot
        const double g0 = rsqrt_(fma(p00, p11, -p10 * p10));
        const double g = __double_as_longlong(p00) > 0 ? g0 : __longlong_as_double(0x7ff8000000000000ll);
        if (NEG) { acc.in = fma(s, g, acc.in); acc.ep += s; } else { acc.ip = fma(s, g, acc.ip); acc.en += s; }
      } else {
        constexpr int DN = 2 * Q - 2;
        const double r0 = rsqrt_(p00);
        const double w = p10 * r0;
        const double r1 = rsqrt_(fma(-w, w, p11));
        const double g = r0 * r1;
        const double kap = -w * g;
        double w0[DN], w1[DN];
#pragma unroll
        for (int a = 0; a < DN; ++a) {
          const double u0 = c[tri(OFF + 2 + a, OFF)], u1 = c[tri(OFF + 2 + a, OFF + 1)];
          w0[a] = u0 * r0;
          w1[a] = fma(u0, kap, u1 * r1);
        }
        double cn[sym(DN)];
#pragma unroll
        for (int a = 0; a < DN; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b)
            cn[tri(a, b)] = fma(-w1[a], w1[b], fma(-w0[a], w0[b], c[tri(OFF + 2 + a, OFF + 2 + b)]));
        Dfs<E, Q - 1, DN, 0, NEG, PAIR>::run(cn, s * g, acc, bad);
        Dfs<E, Q - 1, D, OFF + 2, !NEG, PAIR>::run(c, s, acc, bad);
      }
    } else {
    const T p00 = re_of(c[tri(OFF, OFF)]);
    const T p11 = re_of(c[tri(OFF + 1, OFF + 1)]);
    const E p10 = c[tri(OFF + 1, OFF)];
    const T det = p00 * p11 - norm2(p10);
    bad |= not_positive(det);
    const T g = rsqrt_(det);
    if constexpr (Q == 1) {
      // include leaf s*g with sign (-1)^NEG; exclude leaf s with one more exclusion
      if (NEG) { acc_fpa(acc.in, s, g); acc_add(acc.ep, s); } else { acc_fpa(acc.ip, s, g); acc_add(acc.en, s); }
    } else {
      constexpr int DN = 2 * Q - 2;
      E cn[sym(DN)];
      const T inv = g * g;
      const T q00 = p00 * inv, q11 = p11 * inv;
      const E m10 = neg_(scale_(p10, inv));
#pragma unroll
      for (int a = 0; a < DN; ++a) {
        const E u0 = c[tri(OFF + 2 + a, OFF)], u1 = c[tri(OFF + 2 + a, OFF + 1)];
        const E L0 = lin2(u0, q11, u1, m10);
        const E L1 = lin2(u1, q00, u0, conj_(m10));
#pragma unroll
        for (int b = 0; b < a; ++b) {
          E v = fms_conj(c[tri(OFF + 2 + a, OFF + 2 + b)], L0, c[tri(OFF + 2 + b, OFF)]);
          cn[tri(a, b)] = fms_conj(v, L1, c[tri(OFF + 2 + b, OFF + 1)]);
        }
        E v = fms_conj_re(c[tri(OFF + 2 + a, OFF + 2 + a)], L0, u0);
        cn[tri(a, a)] = fms_conj_re(v, L1, u1);
      }
      Dfs<E, Q - 1, DN, 0, NEG, PAIR>::run(cn, s * g, acc, bad);
      Dfs<E, Q - 1, D, OFF + 2, !NEG, PAIR>::run(c, s, acc, bad);
    }
    }
  }
};

// Register subtree of one node (all Q levels below it): the node's signed sums
// as reduction values and its absolute sum; returns false if a pivot was not
// positive definite (the sums then carry NaN or inf, or the type flagged it).
GBS_HD dd red_diff(double a, double b, dd*) {
  dd r;
  two_sum(a, -b, r.hi, r.lo);
  return r;
}
GBS_HD dd red_diff(const dd& a, const dd& b, dd*) { return a - b; }
GBS_HD td red_diff(const td& a, const td& b, td*) { return a - b; }

// PAIR: inc receives the node's Torontonian (every group's v), exc zero, and
// asum the sum of the group magnitudes.
template <class E, int Q, bool PAIR = false, class Red>
__device__ __forceinline__ bool subtree_sums(const E (&c)[sym(2 * Q)], const typename scale_of<E>::type& s, Red& inc,
                                             Red& exc, double& asum) {
  typedef typename acc_traits<typename real_of<E>::type>::Acc Acc;
  Sums<Acc> a = sums_zero<Acc>();
  bool bad = false;
  Dfs<E, Q, 2 * Q, 0, false, PAIR>::run(c, s, a, bad);
  if constexpr (PAIR) {
    inc = red_diff(a.ip, a.in, (Red*)nullptr);
    exc = red_zero<Red>();
    asum = to_double(a.ep);
    return isfinite(asum) && isfinite(to_double(a.ip));
  } else {
    inc = red_diff(a.ip, a.in, (Red*)nullptr);
    exc = red_diff(a.ep, a.en, (Red*)nullptr);
    asum = sums_total<Acc>::of(a);
    return !bad && isfinite(asum);
  }
}

// Register subtree of one node into per-thread sign-split sums (added to acc);
// false if a pivot was not positive definite.
template <class E, int Q, bool PAIR = false>
__device__ __forceinline__ bool subtree_run(const E (&c)[sym(2 * Q)], const typename scale_of<E>::type& s,
                                            Sums<typename acc_traits<typename real_of<E>::type>::Acc>& a) {
  bool bad = false;
  Dfs<E, Q, 2 * Q, 0, false, PAIR>::run(c, s, a, bad);
  return !bad;
}

// Block reduction of per-thread FP64 sign-split sums (ip, in, ep, en) into one
// double-double partial.  In a plain tree the four sums are non-negative, so a
// warp adds them in FP64 (five rounding levels, relative error <= 5 u each, no
// cancellation); lane 0 then forms inc = ip - in and exc = ep - en exactly
// (TwoSum) and one thread adds the warps' partials in double-double.  This
// keeps the reduction at ~20 FP64 additions per thread instead of the ~110 of
// a double-double warp reduction.  PAIR (cancellation-free last levels): ip
// and in carry the signed group values, ep + en the group magnitudes.
template <bool PAIR>
__device__ __forceinline__ void block_reduce_sums(double ip, double in, double ep, double en, Partial<dd>* out) {
  __shared__ dd s_inc[32], s_exc[32];
  __shared__ double s_abs[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ip += __shfl_down_sync(0xffffffffu, ip, off);
    in += __shfl_down_sync(0xffffffffu, in, off);
    ep += __shfl_down_sync(0xffffffffu, ep, off);
    en += __shfl_down_sync(0xffffffffu, en, off);
  }
  if (lane == 0) {
    s_inc[warp] = red_diff(ip, in, (dd*)nullptr);
    s_exc[warp] = PAIR ? dd_make(0.0) : red_diff(ep, en, (dd*)nullptr);
    s_abs[warp] = PAIR ? ep + en : (ip + in) + (ep + en);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    dd a = s_inc[0], b = s_exc[0];
    double c = s_abs[0];
    for (int w = 1; w < nw; ++w) { a = a + s_inc[w]; b = b + s_exc[w]; c += s_abs[w]; }
    out->inc = a; out->exc = b; out->abs = c;
  }
}

template <class Red>
__device__ __forceinline__ void block_reduce_store(Red inc, Red exc, double asum, Partial<Red>* out) {
  __shared__ Red s_inc[32], s_exc[32];
  __shared__ double s_abs[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    inc = red_add(inc, shfl_down(inc, off));
    exc = red_add(exc, shfl_down(exc, off));
    asum += __shfl_down_sync(0xffffffffu, asum, off);
  }
  if (lane == 0) { s_inc[warp] = inc; s_exc[warp] = exc; s_abs[warp] = asum; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    Red a = s_inc[0], b = s_exc[0];
    double c = s_abs[0];
    for (int w = 1; w < nw; ++w) { a = red_add(a, s_inc[w]); b = red_add(b, s_exc[w]); c += s_abs[w]; }
    out->inc = a; out->exc = b; out->abs = c;
  }
}

// One thread per node with Q undecided modes; depth = n - Q levels above.
template <class E, int Q>
__global__ void __launch_bounds__(128) tree_leaf_kernel(const E* __restrict__ nodes,
                                                        const typename scale_of<E>::type* __restrict__ snode,
                                                        long long count, int depth,
                                                        Partial<typename acc_traits<typename real_of<E>::type>::Red>* partials,
                                                        int* __restrict__ status) {
  typedef typename real_of<E>::type T;
  typedef typename acc_traits<T>::Acc Acc;
  typedef typename acc_traits<T>::Red Red;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Red inc = red_zero<Red>(), exc = red_zero<Red>();
  double asum = 0.0;
  if (node < count) {
    E c[sym(2 * Q)];
#pragma unroll
    for (int e = 0; e < sym(2 * Q); ++e) c[e] = nodes[(long long)e * count + node];
    const typename scale_of<E>::type s = snode[node];
    if (!subtree_sums<E, Q>(c, s, inc, exc, asum)) atomicExch(status, (int)kStatusNotPD);
    // sign of the node: (-1)^(exclusions above) = (-1)^(depth - popcount(node))
    if ((depth - __popcll((unsigned long long)node)) & 1) { inc = red_neg(inc); exc = red_neg(exc); }
  }
  block_reduce_store(inc, exc, asum, partials + blockIdx.x);
}

template <class Red>
__global__ void tree_final_kernel(const Partial<Red>* __restrict__ partials, int nparts, TreeOut* out) {
  Red inc = red_zero<Red>(), exc = red_zero<Red>();
  double asum = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    inc = red_add(inc, partials[i].inc);
    exc = red_add(exc, partials[i].exc);
    asum += partials[i].abs;
  }
  __shared__ Partial<Red> res;
  block_reduce_store(inc, exc, asum, &res);
  __syncthreads();
  if (threadIdx.x == 0) {
    red_store(res.inc, out->inc);
    red_store(res.exc, out->exc);
    out->abs = res.abs;
  }
}

}  // namespace gbs
