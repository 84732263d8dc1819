// Fixed-point multiword numbers on the integer pipe: the "FX" precision.
//
// The subset tree needs ~160-bit arithmetic once the cancellation ratio passes
// ~1e20.  Built from FP64 error-free transformations (triple-double) each
// operation costs ~30 FP64 instructions, and this GPU issues only 2 FP64 FMAs
// per clock per SM, against ~60 32-bit integer multiply-adds and carry-chained
// adds.  fxn<L> holds a two's-complement integer X of L 32-bit limbs (limb 0
// least significant) read as X * 2^(-32 (L-2)): fx = fxn<7> has 160 fraction
// bits, fxw = fxn<8> 192, both a range of +-2^63.  Additions are exact (one
// carry-chained instruction per limb); a product keeps the columns at and
// above the fraction point of the exact 2L-limb product, which leaves an error
// of at most 2L units of the last place, biased low.
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

// fxn<L>: L limbs, L - 2 of them fraction limbs (range +-2^63 in every width).
template <int L>
struct fxn {
  uint32_t w[L];
};
typedef fxn<7> fx;   // 160 fraction bits (GBS_PREC_FX)
typedef fxn<8> fxw;  // 192 fraction bits (GBS_PREC_FXW)

// ------------------------------------------------ carry-chained primitives --
// The carry flag lives between consecutive volatile asm statements of one
// chain; nothing else in these functions touches it.
#ifdef __CUDA_ARCH__
#define GBS_ASM1(op, r, a, b) asm volatile(op " %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b))
#define GBS_ASM2(op, r, a, b, c) asm volatile(op " %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c))
#else
#define GBS_ASM1(op, r, a, b) (r = 0u)
#define GBS_ASM2(op, r, a, b, c) (r = 0u)
#endif
GBS_HD uint32_t add_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("add.cc.u32", r, a, b); return r; }
GBS_HD uint32_t addc_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("addc.cc.u32", r, a, b); return r; }
GBS_HD uint32_t addc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("addc.u32", r, a, b); return r; }
GBS_HD uint32_t sub_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("sub.cc.u32", r, a, b); return r; }
GBS_HD uint32_t subc_cc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("subc.cc.u32", r, a, b); return r; }
GBS_HD uint32_t subc(uint32_t a, uint32_t b) { uint32_t r; GBS_ASM1("subc.u32", r, a, b); return r; }
GBS_HD uint32_t mad_lo_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; GBS_ASM2("mad.lo.cc.u32", r, a, b, c); return r; }
GBS_HD uint32_t madc_lo_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; GBS_ASM2("madc.lo.cc.u32", r, a, b, c); return r; }
GBS_HD uint32_t mad_hi_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; GBS_ASM2("mad.hi.cc.u32", r, a, b, c); return r; }
GBS_HD uint32_t madc_hi_cc(uint32_t a, uint32_t b, uint32_t c) { uint32_t r; GBS_ASM2("madc.hi.cc.u32", r, a, b, c); return r; }
#undef GBS_ASM1
#undef GBS_ASM2

// ---------------------------------------------------------------- basics --
template <int L>
GBS_HD fxn<L> operator+(const fxn<L>& a, const fxn<L>& b) {
  fxn<L> r;
  r.w[0] = add_cc(a.w[0], b.w[0]);
#pragma unroll
  for (int k = 1; k < L - 1; ++k) r.w[k] = addc_cc(a.w[k], b.w[k]);
  r.w[L - 1] = addc(a.w[L - 1], b.w[L - 1]);
  return r;
}
template <int L>
GBS_HD fxn<L> operator-(const fxn<L>& a, const fxn<L>& b) {
  fxn<L> r;
  r.w[0] = sub_cc(a.w[0], b.w[0]);
#pragma unroll
  for (int k = 1; k < L - 1; ++k) r.w[k] = subc_cc(a.w[k], b.w[k]);
  r.w[L - 1] = subc(a.w[L - 1], b.w[L - 1]);
  return r;
}
template <int L>
GBS_HD fxn<L> operator-(const fxn<L>& a) {
  fxn<L> r;
  r.w[0] = sub_cc(0u, a.w[0]);
#pragma unroll
  for (int k = 1; k < L - 1; ++k) r.w[k] = subc_cc(0u, a.w[k]);
  r.w[L - 1] = subc(0u, a.w[L - 1]);
  return r;
}
// x / 2 (arithmetic shift by one bit)
template <int L>
GBS_HD fxn<L> fx_half(const fxn<L>& a) {
  fxn<L> r;
#pragma unroll
  for (int k = 0; k < L - 1; ++k) r.w[k] = (a.w[k] >> 1) | (a.w[k + 1] << 31);
  r.w[L - 1] = (uint32_t)((int32_t)a.w[L - 1] >> 1);
  return r;
}

// ---------------------------------------------------------------- product --
// Window of the unsigned product: columns F to F + L - 1 (F = L - 2 fraction
// limbs).  Low halves of the partial products a_i b_j with i + j >= F and high
// halves with i + j >= F - 1 are summed in two arrays; in either array the
// carry out of row i lands in a column that no earlier row has reached, so one
// add captures it.  The low halves of column F - 1 and everything below are
// dropped: at most 2L units of the last place, always toward -inf.  The
// two's-complement correction subtracts b (resp. a) shifted by L limbs when a
// (resp. b) is negative.
template <int L>
GBS_HD fxn<L> operator*(const fxn<L>& a, const fxn<L>& b) {
  constexpr int F = L - 2, W = L, C0 = F;  // C0: column of word 0
  uint32_t lo[W], hi[W];
#pragma unroll
  for (int k = 0; k < W; ++k) lo[k] = hi[k] = 0u;
#pragma unroll
  for (int i = 0; i < L; ++i) {
    {  // lo(a_i b_j) -> column i + j, for columns C0 .. C0 + W - 1
      const int j0 = (C0 - i) > 0 ? (C0 - i) : 0;
      const int j1 = (C0 + W - 1 - i) < (L - 1) ? (C0 + W - 1 - i) : (L - 1);
      if (j0 <= j1) {
        lo[i + j0 - C0] = mad_lo_cc(a.w[i], b.w[j0], lo[i + j0 - C0]);
#pragma unroll
        for (int j = j0 + 1; j <= j1; ++j) lo[i + j - C0] = madc_lo_cc(a.w[i], b.w[j], lo[i + j - C0]);
        if (i + j1 + 1 - C0 < W) lo[i + j1 + 1 - C0] = addc(0u, 0u);
      }
    }
    {  // hi(a_i b_j) -> column i + j + 1
      const int j0 = (C0 - 1 - i) > 0 ? (C0 - 1 - i) : 0;
      const int j1 = (C0 + W - 2 - i) < (L - 1) ? (C0 + W - 2 - i) : (L - 1);
      if (j0 <= j1) {
        hi[i + j0 + 1 - C0] = mad_hi_cc(a.w[i], b.w[j0], hi[i + j0 + 1 - C0]);
#pragma unroll
        for (int j = j0 + 1; j <= j1; ++j) hi[i + j + 1 - C0] = madc_hi_cc(a.w[i], b.w[j], hi[i + j + 1 - C0]);
        if (i + j1 + 2 - C0 < W) hi[i + j1 + 2 - C0] = addc(0u, 0u);
      }
    }
  }
  fxn<L> r;
  r.w[0] = add_cc(lo[0], hi[0]);
#pragma unroll
  for (int k = 1; k < L - 1; ++k) r.w[k] = addc_cc(lo[k], hi[k]);
  r.w[L - 1] = addc(lo[L - 1], hi[L - 1]);
  // signed correction: result limbs S .. L-1 (column L and up) minus masked limbs
  constexpr int S = L - F;
  const uint32_t ma = (uint32_t)((int32_t)a.w[L - 1] >> 31), mb = (uint32_t)((int32_t)b.w[L - 1] >> 31);
  r.w[S] = sub_cc(r.w[S], b.w[0] & ma);
#pragma unroll
  for (int k = S + 1; k < L - 1; ++k) r.w[k] = subc_cc(r.w[k], b.w[k - S] & ma);
  r.w[L - 1] = subc(r.w[L - 1], b.w[L - 1 - S] & ma);
  r.w[S] = sub_cc(r.w[S], a.w[0] & mb);
#pragma unroll
  for (int k = S + 1; k < L - 1; ++k) r.w[k] = subc_cc(r.w[k], a.w[k - S] & mb);
  r.w[L - 1] = subc(r.w[L - 1], a.w[L - 1 - S] & mb);
  return r;
}

// ----------------------------------------------------------- conversions --
// Exact for |x| < 2^62 down to 2^-(32 (L-2)) (bits below are dropped, toward zero).
template <int L>
GBS_HD fxn<L> fx_from_double(double x) {
  fxn<L> r;
#ifdef __CUDA_ARCH__
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long bits;
  memcpy(&bits, &x, 8);
#endif
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned long long m = (bits & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  const int sh = (e ? e : 1) - 1075 + 32 * (L - 2);  // bit position of m's last bit in X
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const int s = 32 * k - sh;
    const unsigned long long v = s >= 0 ? (s < 64 ? (m >> s) : 0ull) : (s > -64 ? (m << (-s)) : 0ull);
    r.w[k] = (uint32_t)v;
  }
  return (bits >> 63) ? -r : r;
}
template <> GBS_HD fx from_double<fx>(double x) { return fx_from_double<7>(x); }
template <> GBS_HD fxw from_double<fxw>(double x) { return fx_from_double<8>(x); }

// Nearest-ish double (a few units of the last place).
template <int L>
GBS_HD double to_double(const fxn<L>& a) {
  double v = (double)(int32_t)a.w[L - 1];
#pragma unroll
  for (int k = L - 2; k >= 0; --k) v = fma(v, 4294967296.0, (double)a.w[k]);
  return v * (L == 7 ? 0x1p-160 : 0x1p-192);
}
static_assert(sizeof(fx) == 28 && sizeof(fxw) == 32, "fx widths");

// ------------------------------------------------------ tree interface ----
template <int L> GBS_HD fxn<L> fms(const fxn<L>& x, const fxn<L>& a, const fxn<L>& b) { return x - a * b; }
template <int L> GBS_HD fxn<L> fpa(const fxn<L>& x, const fxn<L>& a, const fxn<L>& b) { return x + a * b; }
template <> GBS_HD fx scale_<fx, fx>(const fx& x, const fx& s) { return x * s; }
template <> GBS_HD fxw scale_<fxw, fxw>(const fxw& x, const fxw& s) { return x * s; }
template <> GBS_HD fx conv_entry<fx>(const double& x) { return from_double<fx>(x); }
template <> GBS_HD fxw conv_entry<fxw>(const double& x) { return from_double<fxw>(x); }

// A pivot determinant the fixed-point tree can use: in [2^-20, 2^12), where
// its inverse square root keeps ~150 bits (the resolution is absolute, so the
// relative error of 1/sqrt(x) grows like 2^-(32 (L-2)) x).
template <int L>
GBS_HD bool fx_det_in_range(const fxn<L>& d) {
  return d.w[L - 1] == 0u && d.w[L - 2] < (1u << 12) && (d.w[L - 2] != 0u || d.w[L - 3] >= (1u << 12));
}
template <int L> GBS_HD bool not_positive(const fxn<L>& d) { return !fx_det_in_range(d); }
template <int L> GBS_HD bool is_pos(const fxn<L>& d) { return fx_det_in_range(d); }
template <> constexpr int bad_status<fx>() { return kStatusRange; }
template <> constexpr int bad_status<fxw>() { return kStatusRange; }

// 1/sqrt(x) for x in [2^-20, 2^12): FP64 seed from the top limbs below the
// sign limb, then Newton steps y <- y + y (1 - x y^2) / 2 (53 -> 106 -> 212 bits).
template <int L>
__device__ __forceinline__ fxn<L> rsqrt_(const fxn<L>& x) {
  const double xd = fma((double)x.w[L - 3], 0x1p-32, (double)x.w[L - 2]) + (double)x.w[L - 4] * 0x1p-64;
  fxn<L> y = fx_from_double<L>(rsqrt(xd));
  fxn<L> one;
#pragma unroll
  for (int k = 0; k < L; ++k) one.w[k] = k == L - 2 ? 1u : 0u;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const fxn<L> e = one - x * (y * y);
    y = y + fx_half(y * e);
  }
  return y;
}

// ------------------------------------------------------ sums and reduction --
template <int L> struct acc_traits<fxn<L>> { typedef fxn<L> Acc; typedef fxn<L> Red; };
template <int L> GBS_HD void acc_add(fxn<L>& a, const fxn<L>& x) { a = a + x; }
template <int L> GBS_HD void acc_sub(fxn<L>& a, const fxn<L>& x) { a = a - x; }
template <int L> GBS_HD void acc_fpa(fxn<L>& acc, const fxn<L>& a, const fxn<L>& b) { acc = acc + a * b; }
template <int L> GBS_HD fxn<L> red_diff(const fxn<L>& a, const fxn<L>& b, fxn<L>*) { return a - b; }
template <int L> GBS_HD fxn<L> to_red(const fxn<L>& a, fxn<L>*) { return a; }
template <int L> GBS_HD fxn<L> red_add(const fxn<L>& a, const fxn<L>& b) { return a + b; }
template <int L> GBS_HD fxn<L> red_neg(const fxn<L>& a) { return -a; }
template <> GBS_HD fx red_zero<fx>() { return from_double<fx>(0.0); }
template <> GBS_HD fxw red_zero<fxw>() { return from_double<fxw>(0.0); }
// Three doubles whose sum is the value to ~2^-159 relative (each the nearest
// double of what the previous ones left over; the differences are exact).
template <int L>
GBS_HD void red_store(const fxn<L>& a, double* o) {
  const double x0 = to_double(a);
  const fxn<L> r1 = a - fx_from_double<L>(x0);
  const double x1 = to_double(r1);
  const fxn<L> r2 = r1 - fx_from_double<L>(x1);
  o[0] = x0;
  o[1] = x1;
  o[2] = to_double(r2);
}
template <int L>
__device__ __forceinline__ fxn<L> shfl_down(const fxn<L>& v, int off) {
  fxn<L> r;
#pragma unroll
  for (int k = 0; k < L; ++k) r.w[k] = __shfl_down_sync(0xffffffffu, v.w[k], off);
  return r;
}

}  // namespace gbs
