// Fixed-point multiword numbers on the integer pipe: the "FX" precisions.
//
// The subset tree needs ~160-bit arithmetic once the cancellation ratio passes
// ~1e20.  Built from FP64 error-free transformations (triple-double) each
// operation costs ~30 FP64 instructions, and this GPU issues only 2 FP64 FMAs
// per clock per SM, against ~60 32-bit integer multiply-adds and carry-chained
// adds.  fxn<L, F> holds a two's-complement integer X of L 32-bit limbs (limb 0
// least significant) read as X * 2^(-32 F).  Two widths serve each precision:
// the matrix entries and the scalars derived from them (pivots, determinants,
// inverse square roots) need only 31 integer bits, the running product s of
// pivot factors and the sums of terms need 63:
//   FXN   entries fxn4 = fxn<5, 4>, s and sums fxn4s = fxn<6, 4>  (128 fraction bits)
//   FX    entries fx   = fxn<6, 5>, s and sums fxs   = fxn<7, 5>  (160 fraction bits)
//   FXW   entries fxw  = fxn<7, 6>, s and sums fxws  = fxn<8, 6>  (192 fraction bits)
// Additions are exact (one carry-chained instruction per limb); a product
// keeps the columns at and above the fraction point of the exact 2L-limb
// product, which leaves an error of at most F units of the last place,
// biased low.
//
// Inside the tree every value stays in range when the caller has checked it:
// entries are bounded by the largest eigenvalue of the root, pivot
// determinants by its smallest, and s and the sums by (1 + 1/lambda_min)^n.
// A pivot determinant outside [2^-20, 2^12) is reported (kStatusRange) and
// the caller redoes the tree in triple-double.
//
// Everything here is device code; the host copies exist only so that the
// generic host/device helpers of the tree compile, and are never called.
#pragma once
#include <stdint.h>
#include <string.h>

#include "gbs_tree_driver.cuh"

namespace gbs {

template <int L, int F>
struct fxn {
  static_assert(F >= 3 && L > F, "at least three fraction limbs and one integer limb");
  uint32_t w[L];
};
typedef fxn<5, 4> fxn4;  // FXN entries
typedef fxn<6, 4> fxn4s; // FXN s and sums
typedef fxn<6, 5> fx;    // FX entries
typedef fxn<7, 5> fxs;   // FX s and sums
typedef fxn<7, 6> fxw;   // FXW entries
typedef fxn<8, 6> fxws;  // FXW s and sums

// ------------------------------------------------ carry-chained primitives --
// The carry flag lives between consecutive volatile asm statements of one
// chain; nothing else in these functions touches it.
#ifdef __CUDA_ARCH__
#define GBS_ASM1(op, r, a, b) asm volatile(op " %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b))
#else
#define GBS_ASM1(op, r, a, b) (r = 0u)
#endif
GBS_HD uint32_t add_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("add.cc.u32", r, a, b); return r; }
GBS_HD uint32_t addc_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("addc.cc.u32", r, a, b); return r; }
GBS_HD uint32_t addc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("addc.u32", r, a, b); return r; }
GBS_HD uint32_t sub_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("sub.cc.u32", r, a, b); return r; }
GBS_HD uint32_t subc_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("subc.cc.u32", r, a, b); return r; }
GBS_HD uint32_t subc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("subc.u32", r, a, b); return r; }
#undef GBS_ASM1

// ---------------------------------------------------------------- basics --
template <int L, int F>
GBS_HD fxn<L, F> operator+(const fxn<L, F>& a, const fxn<L, F>& b) {
  fxn<L, F> r;
  r.w[0] = add_cc(a.w[0], b.w[0]);
#pragma unroll
  for (int k = 1; k < L - 1; ++k) r.w[k] = addc_cc(a.w[k], b.w[k]);
  r.w[L - 1] = addc(a.w[L - 1], b.w[L - 1]);
  return r;
}
template <int L, int F>
GBS_HD fxn<L, F> operator-(const fxn<L, F>& a, const fxn<L, F>& b) {
  fxn<L, F> r;
  r.w[0] = sub_cc(a.w[0], b.w[0]);
#pragma unroll
  for (int k = 1; k < L - 1; ++k) r.w[k] = subc_cc(a.w[k], b.w[k]);
  r.w[L - 1] = subc(a.w[L - 1], b.w[L - 1]);
  return r;
}
template <int L, int F>
GBS_HD fxn<L, F> operator-(const fxn<L, F>& a) {
  fxn<L, F> r;
  r.w[0] = sub_cc(0u, a.w[0]);
#pragma unroll
  for (int k = 1; k < L - 1; ++k) r.w[k] = subc_cc(0u, a.w[k]);
  r.w[L - 1] = subc(0u, a.w[L - 1]);
  return r;
}
// x / 2 (arithmetic shift by one bit)
template <int L, int F>
GBS_HD fxn<L, F> fx_half(const fxn<L, F>& a) {
  fxn<L, F> r;
#pragma unroll
  for (int k = 0; k < L - 1; ++k) r.w[k] = (a.w[k] >> 1) | (a.w[k + 1] << 31);
  r.w[L - 1] = (uint32_t)((int32_t)a.w[L - 1] >> 1);
  return r;
}
// The same value with one more integer limb (sign extension).
template <int L, int F>
GBS_HD fxn<L + 1, F> fx_widen(const fxn<L, F>& a) {
  fxn<L + 1, F> r;
#pragma unroll
  for (int k = 0; k < L; ++k) r.w[k] = a.w[k];
  r.w[L] = (uint32_t)((int32_t)a.w[L - 1] >> 31);
  return r;
}

// ---------------------------------------------------------------- product --
// Window of the unsigned product: columns F to F + L - 1, plus a guard column
// F - 1.  Row by row (operand a_i against the limbs of b that reach the
// window), each partial product is added to its column together with the
// running carry as one 64-bit multiply-add, whose high word is the next
// carry; a row's final carry lands in the column one past its last product,
// which no earlier row has reached (rows whose last product is the top
// column drop it: the arithmetic is modulo 2^(32 L)).  Partial products below
// the guard column are not formed and the guard column is dropped: at most F
// units of the last place, always toward -inf.  The two's-complement
// correction subtracts b (resp. a) shifted by L limbs when a (resp. b) is
// negative.
template <int L, int F>
GBS_HD fxn<L, F> operator*(const fxn<L, F>& a, const fxn<L, F>& b) {
  constexpr int W = L, G = F - 1;  // G: column of r[0] (the guard)
  uint32_t r[W + 1];
#pragma unroll
  for (int k = 0; k <= W; ++k) r[k] = 0u;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const int j0 = (G - i) > 0 ? (G - i) : 0;
    const int j1 = (G + W - i) < (L - 1) ? (G + W - i) : (L - 1);
    if (j0 > j1) continue;
    uint32_t carry = 0u;
#pragma unroll
    for (int j = j0; j <= j1; ++j) {
      const unsigned long long t = (unsigned long long)a.w[i] * b.w[j] + r[i + j - G] + carry;
      r[i + j - G] = (uint32_t)t;
      carry = (uint32_t)(t >> 32);
    }
    if (i + j1 + 1 - G <= W) r[i + j1 + 1 - G] = carry;
  }
  fxn<L, F> out;
#pragma unroll
  for (int k = 0; k < L; ++k) out.w[k] = r[k + 1];
  // signed correction: result limbs S .. L-1 (column L and up) minus masked limbs
  constexpr int S = L - F;
  const uint32_t ma = (uint32_t)((int32_t)a.w[L - 1] >> 31), mb = (uint32_t)((int32_t)b.w[L - 1] >> 31);
  if constexpr (S == L - 1) {
    out.w[S] -= (b.w[0] & ma) + (a.w[0] & mb);
  } else {
    out.w[S] = sub_cc(out.w[S], b.w[0] & ma);
#pragma unroll
    for (int k = S + 1; k < L - 1; ++k) out.w[k] = subc_cc(out.w[k], b.w[k - S] & ma);
    out.w[L - 1] = subc(out.w[L - 1], b.w[L - 1 - S] & ma);
    out.w[S] = sub_cc(out.w[S], a.w[0] & mb);
#pragma unroll
    for (int k = S + 1; k < L - 1; ++k) out.w[k] = subc_cc(out.w[k], a.w[k - S] & mb);
    out.w[L - 1] = subc(out.w[L - 1], a.w[L - 1 - S] & mb);
  }
  return out;
}
// s * g: the wide scale type times an entry scalar.
template <int L, int F>
GBS_HD fxn<L + 1, F> operator*(const fxn<L + 1, F>& a, const fxn<L, F>& b) {
  return a * fx_widen(b);
}

// ----------------------------------------------------------- conversions --
// Exact while |x| fits the integer limbs, down to 2^-(32 F) (bits below are
// dropped, toward zero).
template <int L, int F>
GBS_HD fxn<L, F> fx_from_double(double x) {
  fxn<L, F> r;
#ifdef __CUDA_ARCH__
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long bits;
  memcpy(&bits, &x, 8);
#endif
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned long long m = (bits & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  const int sh = (e ? e : 1) - 1075 + 32 * F;  // bit position of m's last bit in X
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const int s = 32 * k - sh;
    const unsigned long long v = s >= 0 ? (s < 64 ? (m >> s) : 0ull) : (s > -64 ? (m << (-s)) : 0ull);
    r.w[k] = (uint32_t)v;
  }
  return (bits >> 63) ? -r : r;
}
template <> GBS_HD fxn4 from_double<fxn4>(double x) { return fx_from_double<5, 4>(x); }
template <> GBS_HD fxn4s from_double<fxn4s>(double x) { return fx_from_double<6, 4>(x); }
template <> GBS_HD fx from_double<fx>(double x) { return fx_from_double<6, 5>(x); }
template <> GBS_HD fxs from_double<fxs>(double x) { return fx_from_double<7, 5>(x); }
template <> GBS_HD fxw from_double<fxw>(double x) { return fx_from_double<7, 6>(x); }
template <> GBS_HD fxws from_double<fxws>(double x) { return fx_from_double<8, 6>(x); }

// Nearest-ish double (a few units of the last place).
template <int L, int F>
GBS_HD double to_double(const fxn<L, F>& a) {
  double v = (double)(int32_t)a.w[L - 1];
#pragma unroll
  for (int k = L - 2; k >= 0; --k) v = fma(v, 4294967296.0, (double)a.w[k]);
  return v * (F == 4 ? 0x1p-128 : F == 5 ? 0x1p-160 : 0x1p-192);
}
static_assert(sizeof(fxn4) == 20 && sizeof(fxn4s) == 24 && sizeof(fx) == 24 && sizeof(fxs) == 28 &&
                  sizeof(fxw) == 28 && sizeof(fxws) == 32,
              "fx widths");

// ------------------------------------------------------ tree interface ----
template <int L, int F> GBS_HD fxn<L, F> fms(const fxn<L, F>& x, const fxn<L, F>& a, const fxn<L, F>& b) {
  return x - a * b;
}
template <int L, int F> GBS_HD fxn<L, F> fpa(const fxn<L, F>& x, const fxn<L, F>& a, const fxn<L, F>& b) {
  return x + a * b;
}
template <> GBS_HD fxn4 scale_<fxn4, fxn4>(const fxn4& x, const fxn4& s) { return x * s; }
template <> GBS_HD fx scale_<fx, fx>(const fx& x, const fx& s) { return x * s; }
template <> GBS_HD fxw scale_<fxw, fxw>(const fxw& x, const fxw& s) { return x * s; }
template <> GBS_HD fxn4 conv_entry<fxn4>(const double& x) { return from_double<fxn4>(x); }
template <> GBS_HD fx conv_entry<fx>(const double& x) { return from_double<fx>(x); }
template <> GBS_HD fxw conv_entry<fxw>(const double& x) { return from_double<fxw>(x); }
template <> struct scale_of<fxn4> { typedef fxn4s type; };
template <> struct scale_of<fx> { typedef fxs type; };
template <> struct scale_of<fxw> { typedef fxws type; };

// A pivot determinant the fixed-point tree can use: in [2^-20, 2^12), where
// its inverse square root keeps ~150 bits (the resolution is absolute, so the
// relative error of 1/sqrt(x) grows like 2^-(32 F) x).
template <int L, int F>
GBS_HD bool fx_det_in_range(const fxn<L, F>& d) {
  bool high_zero = true;
#pragma unroll
  for (int k = F + 1; k < L; ++k) high_zero &= d.w[k] == 0u;
  return high_zero && d.w[F] < (1u << 12) && (d.w[F] != 0u || d.w[F - 1] >= (1u << 12));
}
template <int L, int F> GBS_HD bool not_positive(const fxn<L, F>& d) { return !fx_det_in_range(d); }
template <int L, int F> GBS_HD bool is_pos(const fxn<L, F>& d) { return fx_det_in_range(d); }
// Fixed-point trees run only on matrices the host has bounded (positive definite).
template <int L, int F> GBS_HD bool lead_pos(const fxn<L, F>&) { return true; }
template <> constexpr int bad_status<fxn4>() { return kStatusRange; }
template <> struct level_min_blocks<fxn4> { static const int value = 4; };
template <> struct level_park<fxn4> { static const bool value = true; };
template <> constexpr int bad_status<fx>() { return kStatusRange; }
template <> struct level_min_blocks<fx> { static const int value = 4; };
template <> struct level_park<fx> { static const bool value = true; };
template <> struct level_park<fxw> { static const bool value = true; };
template <int L, int F> struct node_words<fxn<L, F>> { static const int value = L; };
template <int L, int F> struct leaf_min_blocks<fxn<L, F>> { static const int value = 4; };
template <> struct level_min_blocks<fxw> { static const int value = 3; };
template <> constexpr int bad_status<fxw>() { return kStatusRange; }

// a * b where b >= 0 has nonzero limbs only in [JLO, JHI] (and, when ILO/IHI
// are given, a >= 0 only in [ILO, IHI]), for the inverse square root's short
// operands: the general product's rows and guard column restricted to those
// rows and columns (the carry of row i still lands in column i + JHI + 1, which
// no earlier row reached), then the one correction a negative a needs.
template <int JLO, int JHI, int L, int F, int ILO = 0, int IHI = L - 1>
__device__ __forceinline__ fxn<L, F> mul_short(const fxn<L, F>& a, const fxn<L, F>& b) {
  constexpr int W = L, G = F - 1;
  uint32_t r[W + 1];
#pragma unroll
  for (int k = 0; k <= W; ++k) r[k] = 0u;
#pragma unroll
  for (int i = ILO; i <= IHI; ++i) {
    const int j0 = (G - i) > JLO ? (G - i) : JLO;
    const int j1 = (G + W - i) < JHI ? (G + W - i) : JHI;
    if (j0 > j1) continue;
    uint32_t carry = 0u;
#pragma unroll
    for (int j = j0; j <= j1; ++j) {
      const unsigned long long t = (unsigned long long)a.w[i] * b.w[j] + r[i + j - G] + carry;
      r[i + j - G] = (uint32_t)t;
      carry = (uint32_t)(t >> 32);
    }
    if (i + j1 + 1 - G <= W) r[i + j1 + 1 - G] = carry;
  }
  fxn<L, F> out;
#pragma unroll
  for (int k = 0; k < L; ++k) out.w[k] = r[k + 1];
  constexpr int S = L - F;
  const uint32_t ma = (uint32_t)((int32_t)a.w[L - 1] >> 31);
  out.w[S] = sub_cc(out.w[S], b.w[0] & ma);
#pragma unroll
  for (int k = S + 1; k < L - 1; ++k) out.w[k] = subc_cc(out.w[k], b.w[k - S] & ma);
  out.w[L - 1] = subc(out.w[L - 1], b.w[L - 1 - S] & ma);
  return out;
}

// The value of a float (exact: 24 significant bits placed in the limbs).
template <int L, int F>
__device__ __forceinline__ fxn<L, F> fx_from_float(float v) {
  const uint32_t bits = __float_as_uint(v);
  const int e = (int)((bits >> 23) & 0xffu);
  const uint32_t m = e ? ((bits & 0x7fffffu) | 0x800000u) : 0u;  // no subnormal reaches here
  const int sh = e - 150 + 32 * F;                              // bit position of m's last bit in X
  fxn<L, F> r;
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const int s = 32 * k - sh;
    r.w[k] = s >= 0 ? (s < 32 ? m >> s : 0u) : (s > -32 ? m << (-s) : 0u);
  }
  return (bits >> 31) ? -r : r;
}

// 1/sqrt(x) for x in [2^-20, 2^12), on the integer pipe apart from an FP32
// seed.  Seed: the single-precision inverse square root of the float of x's
// two leading limbs (from the integer limb, or from the first fraction limb
// when x < 1; the limbs left out change x by less than 2^-32 relative), with
// a relative error below 2^-21; when the seed rounded
// to 12 significant bits squares exactly to 1/x in single precision it is
// taken instead, so that exact cases (x = 1, 1/4, 4, ...) stay exact.  The
// seed lies in (2^-6, 2^11), i.e. in limbs F-1 .. F.  Then two third-order
// steps y <- y (1 + e/2 + 3 e^2 / 8), e = 1 - x y^2:
//   1. y0^2 is exact (48 bits), e^2 comes from the float of e (|e| < 2^-20);
//      the result, cut to limbs F-2 .. F (2^-64 resolution), has |e| < 2^-55;
//   2. y1^2 is exact (192 bits), e^2 is a short product of |e| cut to limbs
//      F-5 .. F-2; the remaining error 5|e|^3/16 is below 2^-165 relative.
// Every product has a short nonnegative factor (mul_short).
template <int L, int F>
__device__ __forceinline__ fxn<L, F> rsqrt_(const fxn<L, F>& x) {
  fxn<L, F> one;
#pragma unroll
  for (int k = 0; k < L; ++k) one.w[k] = k == F ? 1u : 0u;
  const float xf = x.w[F] ? __ull2float_rn(((unsigned long long)x.w[F] << 32) | x.w[F - 1]) * 0x1p-32f
                          : __ull2float_rn(((unsigned long long)x.w[F - 1] << 32) | x.w[F - 2]) * 0x1p-64f;
  float yf = rsqrtf(xf);
  const float ys = __uint_as_float((__float_as_uint(yf) + 0x800u) & ~0xfffu);
  if (fmaf(xf * ys, ys, -1.0f) == 0.0f) yf = ys;
  const fxn<L, F> y0 = fx_from_float<L, F>(yf);
  // step 1
  const fxn<L, F> y0sq = mul_short<F - 1, F, L, F, F - 1, F>(y0, y0);
  const fxn<L, F> e0 = one - mul_short<F - 2, F>(x, y0sq);
  const float e0f = __ll2float_rn((long long)(((unsigned long long)e0.w[F - 1] << 32) | e0.w[F - 2])) * 0x1p-64f;
  const fxn<L, F> c0 = fx_half(e0) + fx_from_float<L, F>(0.375f * e0f * e0f);
  fxn<L, F> y1 = y0 + mul_short<F - 1, F>(c0, y0);
#pragma unroll
  for (int k = 0; k < F - 2; ++k) y1.w[k] = 0u;
  // step 2
  constexpr int ELO = F - 5 > 0 ? F - 5 : 0;
  const fxn<L, F> y1sq = mul_short<F - 2, F, L, F, F - 2, F>(y1, y1);
  const fxn<L, F> e1 = one - mul_short<F - 4, F>(x, y1sq);
  const bool neg = (int32_t)e1.w[L - 1] < 0;
  fxn<L, F> ae = neg ? -e1 : e1;
#pragma unroll
  for (int k = 0; k < L; ++k)
    if (k < ELO || k > F - 2) ae.w[k] = 0u;
  const fxn<L, F> esq = mul_short<ELO, F - 2, L, F, ELO, F - 2>(ae, ae);
  const fxn<L, F> q = fx_half(fx_half(esq));
  const fxn<L, F> c1 = fx_half(e1) + (q + fx_half(q));  // e/2 + 3 e^2 / 8
  return y1 + mul_short<F - 2, F>(c1, y1);
}

// ------------------------------------------------------ sums and reduction --
// The four sign-split sums are exact and non-negative: add them, convert once.
template <int L, int F>
struct sums_total<fxn<L, F>> {
  static GBS_HD double of(const Sums<fxn<L, F>>& a) { return to_double((a.ip + a.in) + (a.ep + a.en)); }
};
template <> struct acc_traits<fxn4> { typedef fxn4s Acc; typedef fxn4s Red; };
template <> struct acc_traits<fx> { typedef fxs Acc; typedef fxs Red; };
template <> struct acc_traits<fxw> { typedef fxws Acc; typedef fxws Red; };
template <int L, int F> GBS_HD void acc_add(fxn<L, F>& a, const fxn<L, F>& x) { a = a + x; }
template <int L, int F>
GBS_HD void acc_fpa(fxn<L + 1, F>& acc, const fxn<L + 1, F>& s, const fxn<L, F>& g) { acc = acc + s * g; }
template <int L, int F> GBS_HD fxn<L, F> red_diff(const fxn<L, F>& a, const fxn<L, F>& b, fxn<L, F>*) { return a - b; }
template <int L, int F> GBS_HD fxn<L, F> red_add(const fxn<L, F>& a, const fxn<L, F>& b) { return a + b; }
template <int L, int F> GBS_HD fxn<L, F> red_neg(const fxn<L, F>& a) { return -a; }
template <> GBS_HD fxn4s red_zero<fxn4s>() { return from_double<fxn4s>(0.0); }
template <> GBS_HD fxs red_zero<fxs>() { return from_double<fxs>(0.0); }
template <> GBS_HD fxws red_zero<fxws>() { return from_double<fxws>(0.0); }
// Three doubles whose sum is the value to ~2^-159 relative (each the nearest
// double of what the previous ones left over; the differences are exact).
template <int L, int F>
GBS_HD void red_store(const fxn<L, F>& a, double* o) {
  const double x0 = to_double(a);
  const fxn<L, F> r1 = a - fx_from_double<L, F>(x0);
  const double x1 = to_double(r1);
  const fxn<L, F> r2 = r1 - fx_from_double<L, F>(x1);
  o[0] = x0;
  o[1] = x1;
  o[2] = to_double(r2);
}
template <int L, int F>
__device__ __forceinline__ fxn<L, F> shfl_down(const fxn<L, F>& v, int off) {
  fxn<L, F> r;
#pragma unroll
  for (int k = 0; k < L; ++k) r.w[k] = __shfl_down_sync(0xffffffffu, v.w[k], off);
  return r;
}

}  // namespace gbs
