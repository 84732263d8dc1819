// Fixed-point multiword numbers on the integer pipe: the "FX" precision.
//
// The subset tree needs ~160-bit arithmetic once the cancellation ratio passes
// ~1e20.  Built from FP64 error-free transformations (triple-double) each
// operation costs ~30 FP64 instructions, and this GPU issues only 2 FP64 FMAs
// per clock per SM, against ~60 32-bit integer multiply-adds and carry-chained
// adds.  fx holds a two's-complement integer X of kFxL 32-bit limbs (limb 0
// least significant) read as X * 2^(-32 kFxF): 160 fraction bits and a range
// of +-2^63.  Additions are exact (one carry-chained instruction per limb);
// a product keeps the columns at and above the fraction point of the exact
// 448-bit product (partial products a_i b_j with i + j >= kFxF - 2), which
// leaves an error of at most two units of 2^-160, biased low.
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

constexpr int kFxL = 7;  // limbs
constexpr int kFxF = 5;  // fraction limbs

struct fx {
  uint32_t w[kFxL];
};

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
GBS_HD fx operator+(const fx& a, const fx& b) {
  fx r;
  r.w[0] = add_cc(a.w[0], b.w[0]);
#pragma unroll
  for (int k = 1; k < kFxL - 1; ++k) r.w[k] = addc_cc(a.w[k], b.w[k]);
  r.w[kFxL - 1] = addc(a.w[kFxL - 1], b.w[kFxL - 1]);
  return r;
}
GBS_HD fx operator-(const fx& a, const fx& b) {
  fx r;
  r.w[0] = sub_cc(a.w[0], b.w[0]);
#pragma unroll
  for (int k = 1; k < kFxL - 1; ++k) r.w[k] = subc_cc(a.w[k], b.w[k]);
  r.w[kFxL - 1] = subc(a.w[kFxL - 1], b.w[kFxL - 1]);
  return r;
}
GBS_HD fx operator-(const fx& a) {
  fx r;
  r.w[0] = sub_cc(0u, a.w[0]);
#pragma unroll
  for (int k = 1; k < kFxL - 1; ++k) r.w[k] = subc_cc(0u, a.w[k]);
  r.w[kFxL - 1] = subc(0u, a.w[kFxL - 1]);
  return r;
}
// x / 2 (arithmetic shift by one bit)
GBS_HD fx fx_half(const fx& a) {
  fx r;
#pragma unroll
  for (int k = 0; k < kFxL - 1; ++k) r.w[k] = (a.w[k] >> 1) | (a.w[k + 1] << 31);
  r.w[kFxL - 1] = (uint32_t)((int32_t)a.w[kFxL - 1] >> 1);
  return r;
}

// ---------------------------------------------------------------- product --
// Window of the unsigned product: columns kFxF - 1 (a guard column whose only
// use is its carry) to kFxF + kFxL - 1.  Low and high halves of the partial
// products are summed in two arrays; in either array the carry out of row i
// lands in a column that no earlier row has reached, so one add captures it.
// The two's-complement correction subtracts b (resp. a) shifted by kFxL limbs
// when a (resp. b) is negative.
GBS_HD fx operator*(const fx& a, const fx& b) {
  constexpr int L = kFxL, F = kFxF, W = L + 1, C0 = F - 1;  // C0: column of word 0
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
  fx r;
  (void)add_cc(lo[0], hi[0]);
#pragma unroll
  for (int k = 0; k < L - 1; ++k) r.w[k] = addc_cc(lo[k + 1], hi[k + 1]);
  r.w[L - 1] = addc(lo[L], hi[L]);
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
// Exact for |x| < 2^62 down to 2^-160 (bits below are dropped, toward zero).
template <>
GBS_HD fx from_double<fx>(double x) {
  fx r;
#ifdef __CUDA_ARCH__
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long bits;
  memcpy(&bits, &x, 8);
#endif
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned long long m = (bits & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  const int sh = (e ? e : 1) - 1075 + 32 * kFxF;  // bit position of m's last bit in X
#pragma unroll
  for (int k = 0; k < kFxL; ++k) {
    const int s = 32 * k - sh;
    const unsigned long long v = s >= 0 ? (s < 64 ? (m >> s) : 0ull) : (s > -64 ? (m << (-s)) : 0ull);
    r.w[k] = (uint32_t)v;
  }
  return (bits >> 63) ? -r : r;
}

// Nearest-ish double (a few units of the last place).
GBS_HD double to_double(const fx& a) {
  double v = (double)(int32_t)a.w[kFxL - 1];
#pragma unroll
  for (int k = kFxL - 2; k >= 0; --k) v = fma(v, 4294967296.0, (double)a.w[k]);
  return v * 0x1p-160;
}
static_assert(kFxF == 5, "to_double scales by 2^-(32 kFxF)");

// ------------------------------------------------------ tree interface ----
GBS_HD fx fms(const fx& x, const fx& a, const fx& b) { return x - a * b; }
GBS_HD fx fpa(const fx& x, const fx& a, const fx& b) { return x + a * b; }
template <>
GBS_HD fx scale_<fx, fx>(const fx& x, const fx& s) { return x * s; }
template <>
GBS_HD fx conv_entry<fx>(const double& x) { return from_double<fx>(x); }

// A pivot determinant the fixed-point tree can use: in [2^-20, 2^12), where
// its inverse square root keeps ~150 bits (the resolution is absolute, so the
// relative error of 1/sqrt(x) grows like 2^-160 x).
GBS_HD bool fx_det_in_range(const fx& d) {
  return d.w[6] == 0u && d.w[5] < (1u << 12) && (d.w[5] != 0u || d.w[4] >= (1u << 12));
}
static_assert(kFxL == 7 && kFxF == 5, "limb indices of fx_det_in_range");
GBS_HD bool not_positive(const fx& d) { return !fx_det_in_range(d); }
template <> constexpr int bad_status<fx>() { return kStatusRange; }
GBS_HD bool is_pos(const fx& d) { return fx_det_in_range(d); }

// 1/sqrt(x) for x in [2^-20, 2^12): FP64 seed from the top three limbs, then
// two Newton steps y <- y + y (1 - x y^2) / 2 (53 -> 106 -> 160+ bits).
__device__ __forceinline__ fx rsqrt_(const fx& x) {
  const double xd = fma((double)x.w[4], 0x1p-32, (double)x.w[5]) + (double)x.w[3] * 0x1p-64;
  fx y = from_double<fx>(rsqrt(xd));
  fx one;
#pragma unroll
  for (int k = 0; k < kFxL; ++k) one.w[k] = k == kFxF ? 1u : 0u;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const fx e = one - x * (y * y);
    y = y + fx_half(y * e);
  }
  return y;
}

// ------------------------------------------------------ sums and reduction --
template <> struct acc_traits<fx> { typedef fx Acc; typedef fx Red; };
GBS_HD void acc_add(fx& a, const fx& x) { a = a + x; }
GBS_HD void acc_sub(fx& a, const fx& x) { a = a - x; }
GBS_HD void acc_fpa(fx& acc, const fx& a, const fx& b) { acc = acc + a * b; }
GBS_HD fx red_diff(const fx& a, const fx& b, fx*) { return a - b; }
GBS_HD fx to_red(const fx& a, fx*) { return a; }
GBS_HD fx red_add(const fx& a, const fx& b) { return a + b; }
GBS_HD fx red_neg(const fx& a) { return -a; }
template <> GBS_HD fx red_zero<fx>() { return from_double<fx>(0.0); }
// Three doubles whose sum is the value to ~2^-159 relative (each the nearest
// double of what the previous ones left over; the differences are exact).
GBS_HD void red_store(const fx& a, double* o) {
  const double x0 = to_double(a);
  const fx r1 = a - from_double<fx>(x0);
  const double x1 = to_double(r1);
  const fx r2 = r1 - from_double<fx>(x1);
  o[0] = x0;
  o[1] = x1;
  o[2] = to_double(r2);
}
__device__ __forceinline__ fx shfl_down(const fx& v, int off) {
  fx r;
#pragma unroll
  for (int k = 0; k < kFxL; ++k) r.w[k] = __shfl_down_sync(0xffffffffu, v.w[k], off);
  return r;
}

}  // namespace gbs
