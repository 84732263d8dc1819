// Device number types for the subset-determinant tree.
//
// The Torontonian's alternating sum cancels by a factor kappa = sum|t| / |Tor|
// that reaches 1e20 and beyond for 20+ clicks, so the per-term arithmetic comes
// in several widths:
//   double          FP64 (the throughput kernel)
//   dd              double-double, ~106 bits
//   td              triple-double, ~159 bits
//   float           FP32, only to measure where it breaks down
// and each can be real (symmetric matrices in the paper's x/p basis) or
// complex (Hermitian matrices in the a/a^+ basis).
//
// The extended types are unevaluated sums of doubles built from error-free
// transformations: TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker 1971) and
// TwoProd by fused multiply-add.  Addition is the "sloppy" kind: its error is
// bounded relative to the operands, which is what the tree needs (entries and
// terms are O(1); the final sum's cancellation is paid for by the width).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#define GBS_HD __host__ __device__ __forceinline__

namespace gbs {

// ------------------------------------------------------------- EFTs ------
GBS_HD void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
GBS_HD void fast_two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  e = b - (s - a);
}
GBS_HD void two_prod(double a, double b, double& p, double& e) {
  p = a * b;
  e = fma(a, b, -p);
}

// ---------------------------------------------------------- double-double --
struct dd {
  double hi, lo;
};
GBS_HD dd dd_make(double a) { return dd{a, 0.0}; }
GBS_HD dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
GBS_HD dd operator+(dd a, dd b) {
  double s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  dd r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
GBS_HD dd operator-(dd a, dd b) { return a + (-b); }
GBS_HD dd operator*(dd a, dd b) {
  double p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fma(a.hi, b.lo, e);
  e = fma(a.lo, b.hi, e);
  dd r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
GBS_HD dd operator*(dd a, double b) {
  double p, e;
  two_prod(a.hi, b, p, e);
  e = fma(a.lo, b, e);
  dd r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
GBS_HD dd operator+(dd a, double b) {
  double s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  dd r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
// x - a*b
GBS_HD dd fms(dd x, dd a, dd b) { return x - a * b; }
GBS_HD dd fpa(dd x, dd a, dd b) { return x + a * b; }
GBS_HD double to_double(dd a) { return a.hi + a.lo; }

// 1/sqrt(a) for a > 0: one Newton step x + x(1 - a x^2)/2 from the FP64 value
// takes the ~52 correct bits of the start to ~104.
__device__ __forceinline__ dd rsqrt_(dd a) {
  double x0 = rsqrt(a.hi);
  dd x = dd_make(x0);
  dd r = dd_make(1.0) - a * (x * x);
  return x + (x * r) * 0.5;
}

// ---------------------------------------------------------- triple-double --
struct td {
  double x0, x1, x2;
};
GBS_HD td td_make(double a) { return td{a, 0.0, 0.0}; }
GBS_HD td operator-(td a) { return td{-a.x0, -a.x1, -a.x2}; }

// Re-packing of x0 + x1 + x2 (roughly decreasing, possibly overlapping after
// a cancellation) into three words: two exact TwoSum steps from the top.
GBS_HD td td_pack(double x0, double x1, double x2) {
  double a, b, c, d;
  two_sum(x0, x1, a, b);
  two_sum(b, x2, c, d);
  return td{a, c, d};
}
// Sloppy triple-double addition: the error is bounded relative to the
// operands (about 2^-155 max(|a|, |b|)), which is what the tree needs.
GBS_HD td operator+(td a, td b) {
  double s0, e0, s1, e1;
  two_sum(a.x0, b.x0, s0, e0);
  two_sum(a.x1, b.x1, s1, e1);
  const double t2 = (a.x2 + b.x2) + e1;
  two_sum(s1, e0, s1, e0);
  return td_pack(s0, s1, t2 + e0);
}
GBS_HD td operator-(td a, td b) { return a + (-b); }
GBS_HD td operator*(td a, td b) {
  double p0, q0, p1, q1, p2, q2;
  two_prod(a.x0, b.x0, p0, q0);  // weight 1
  two_prod(a.x0, b.x1, p1, q1);  // weight 2^-53
  two_prod(a.x1, b.x0, p2, q2);  // weight 2^-53
  double t = fma(a.x0, b.x2, fma(a.x1, b.x1, a.x2 * b.x0)) + (q1 + q2);  // weight 2^-106
  double s1, e1, e2;
  two_sum(p1, p2, s1, e1);
  two_sum(s1, q0, s1, e2);
  return td_pack(p0, s1, t + (e1 + e2));
}
GBS_HD td operator*(td a, double b) {
  double p0, q0, p1, q1;
  two_prod(a.x0, b, p0, q0);
  two_prod(a.x1, b, p1, q1);
  double s1, e1;
  two_sum(p1, q0, s1, e1);
  return td_pack(p0, s1, fma(a.x2, b, q1) + e1);
}
GBS_HD td operator+(td a, double b) { return a + td_make(b); }
GBS_HD td fms(td x, td a, td b) { return x - a * b; }
GBS_HD td fpa(td x, td a, td b) { return x + a * b; }
GBS_HD double to_double(td a) { return a.x0 + (a.x1 + a.x2); }
__device__ __forceinline__ td rsqrt_(td a) {
  // Two Newton steps: 52 -> 104 -> ~159 bits.
  td x = td_make(rsqrt(a.x0));
  for (int it = 0; it < 2; ++it) {
    td r = td_make(1.0) - a * (x * x);
    x = x + (x * r) * 0.5;
  }
  return x;
}

// ------------------------------------------ FP64 inverse square root -----
// 1/sqrt(x) for double x with no FP64 instruction at all.  On this GPU the
// FP64 pipe issues 2 fused multiply-adds per clock per SM against 128 FP32
// operations and ~64 32-bit integer operations, so the whole routine runs off
// that pipe:
//   1. x = M 2^(ex - 52) (M the 53-bit significand) is written as x' 2^(2k),
//      x' = M 2^(r - 52) in [1, 4), r = ex mod 2; the leading 24 bits of x'
//      become a float xf (integer ops);
//   2. yf = rsqrtf(xf) = my 2^(ey - 23) (the FP32 special-function unit,
//      relative error below 2^-21 with the truncation of x' included);
//   3. one Newton-Raphson step of the third order (the Taylor series of
//      (1 - e)^(-1/2) to e^2), y = y0 (1 + e/2 + 3 e^2/8), y0 = yf 2^-k, in
//      integer arithmetic:
//        x' yf^2 = M my^2 2^-sh, sh = 98 - r - 2 ey, so D = 2^sh - M my^2 (a
//        128-bit difference, exact) gives E = e 2^64 = floor(D 2^(64 - sh)),
//        |E| < 2^45 (|e| < 2^-19);
//        F = (e/2 + 3 e^2/8) 2^64 = E/2 + 3 (E^2 / 2^64) / 8;
//        Y = my (2^64 + F), an 89-bit integer, rounded to 53 bits (half up) is
//        the significand of y = Y 2^(ey - 87 - k).
// Truncations of E and F cost at most a few units of 2^-64 and the dropped
// 5 e^3/16 stays below 2^-55, so the result is within 0.51 ulp.  Non-positive,
// subnormal, inf and NaN inputs give NaN.
__device__ __forceinline__ double rsqrt_i64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int eb = (int)(hi >> 20);  // sign and biased exponent (>= 0x800 for x < 0)
  const bool ok = (unsigned)(eb - 1) < 0x7feu;
  const int ex = eb - 1023;
  const int r = ex & 1;
  const int k = ex >> 1;
  const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
  const float xf = __uint_as_float(((unsigned)(127 + r) << 23) | ((hi & 0x000fffffu) << 3) | ((unsigned)b >> 29));
  const unsigned yb = __float_as_uint(rsqrtf(xf));
  const unsigned long long my = (yb & 0x7fffffu) | 0x800000u;
  const int ey = (int)(yb >> 23) - 127;
  const int sh = 98 - r - 2 * ey;  // in [96, 104] for any seed in (2^-3, 2)
  const unsigned long long P = my * my;
  const unsigned long long qlo = M * P, qhi = __umul64hi(M, P);
  const unsigned long long dlo = 0ull - qlo;
  const long long dhi = (long long)((1ull << (sh - 64)) - qhi - (qlo != 0ull));
  const long long E = (long long)(((unsigned long long)dhi << (128 - sh)) + (dlo >> (sh - 64)));
  const unsigned long long aE = (unsigned long long)(E < 0 ? -E : E);
  const long long F = (E >> 1) + (long long)((3ull * __umul64hi(aE, aE)) >> 3);
  const unsigned long long aF = (unsigned long long)(F < 0 ? -F : F);
  const unsigned long long tlo = my * aF, thi = __umul64hi(my, aF);
  unsigned long long ylo, yhi;
  if (F >= 0) {
    ylo = tlo;
    yhi = my + thi;
  } else {
    ylo = 0ull - tlo;
    yhi = my - thi - (tlo != 0ull);
  }
  const int lead = 127 - __clzll((long long)yhi);  // bit index of Y's leading one (86..88)
  const int s = lead - 52;                          // 34..36
  const unsigned long long m53 = ((yhi << (64 - s)) | (ylo >> s)) + ((ylo >> (s - 1)) & 1ull);
  const long long bits = ((long long)(lead + ey - 87 - k + 1022) << 52) + (long long)m53;
  return ok ? __longlong_as_double(bits) : __longlong_as_double(0x7ff8000000000000ll);
}

// -------------------------------------------------------- plain types -----
GBS_HD double fms(double x, double a, double b) { return fma(-a, b, x); }
GBS_HD double fpa(double x, double a, double b) { return fma(a, b, x); }
GBS_HD float fms(float x, float a, float b) { return fmaf(-a, b, x); }
GBS_HD float fpa(float x, float a, float b) { return fmaf(a, b, x); }
GBS_HD double to_double(double a) { return a; }
GBS_HD double to_double(float a) { return (double)a; }
__device__ __forceinline__ double rsqrt_(double a) { return rsqrt_i64(a); }
__device__ __forceinline__ float rsqrt_(float a) { return rsqrtf(a); }

template <class T> GBS_HD T from_double(double a);
template <> GBS_HD double from_double<double>(double a) { return a; }
template <> GBS_HD float from_double<float>(double a) { return (float)a; }
template <> GBS_HD dd from_double<dd>(double a) { return dd_make(a); }
template <> GBS_HD td from_double<td>(double a) { return td_make(a); }

// ----------------------------------------------------------- complex ------
template <class T>
struct cplx {
  T re, im;
};

// Entry types of the tree: T (real symmetric) or cplx<T> (complex Hermitian).
// The functions below give both the same interface.
template <class T> GBS_HD T re_of(const T& x) { return x; }
template <class T> GBS_HD T re_of(const cplx<T>& x) { return x.re; }

// |x|^2
template <class T> GBS_HD T norm2(const T& x) { return x * x; }
template <class T> GBS_HD T norm2(const cplx<T>& x) { return fpa(x.re * x.re, x.im, x.im); }

// x - a * conj(b)
template <class T> GBS_HD T fms_conj(const T& x, const T& a, const T& b) { return fms(x, a, b); }
template <class T> GBS_HD cplx<T> fms_conj(const cplx<T>& x, const cplx<T>& a, const cplx<T>& b) {
  cplx<T> r;
  r.re = fms(fms(x.re, a.re, b.re), a.im, b.im);
  r.im = fpa(fms(x.im, a.im, b.re), a.re, b.im);
  return r;
}
// Re(x - a * conj(b)) as a real entry (diagonal of a Hermitian update)
template <class T> GBS_HD T fms_conj_re(const T& x, const T& a, const T& b) { return fms(x, a, b); }
template <class T> GBS_HD cplx<T> fms_conj_re(const cplx<T>& x, const cplx<T>& a, const cplx<T>& b) {
  cplx<T> r;
  r.re = fms(fms(x.re, a.re, b.re), a.im, b.im);
  r.im = from_double<T>(0.0);
  return r;
}
// a * s (s real) + b * w (w general):  used for L = u P^-1
template <class T> GBS_HD T lin2(const T& a, const T& s, const T& b, const T& w) { return fpa(a * s, b, w); }
template <class T>
GBS_HD cplx<T> lin2(const cplx<T>& a, const T& s, const cplx<T>& b, const cplx<T>& w) {
  cplx<T> r;
  r.re = fms(fpa(a.re * s, b.re, w.re), b.im, w.im);
  r.im = fpa(fpa(a.im * s, b.re, w.im), b.im, w.re);
  return r;
}
template <class T> GBS_HD T conj_(const T& x) { return x; }
template <class T> GBS_HD cplx<T> conj_(const cplx<T>& x) { return cplx<T>{x.re, -x.im}; }
template <class T> GBS_HD T neg_(const T& x) { return -x; }
template <class T> GBS_HD cplx<T> neg_(const cplx<T>& x) { return cplx<T>{-x.re, -x.im}; }

template <class E> struct real_of { typedef E type; };
template <class T> struct real_of<cplx<T>> { typedef T type; };

template <class E> struct is_cplx { static const bool value = false; };
template <class T> struct is_cplx<cplx<T>> { static const bool value = true; };

}  // namespace gbs
