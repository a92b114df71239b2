// Double-float ("dd") arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi)/2, which carries a 48-bit significand (unit roundoff about 2^-47) in
// FP32's exponent range.  Built from the error-free transformations of Knuth and Dekker
// (two_sum, fast_two_sum, two_prod via fused multiply-add), composed as in Shewchuk (1997) and
// Hida, Li and Bailey's double-double arithmetic, restated here for FP32 components.
//
// Why: on this GPU the FP64 pipe issues at 1/61 of the FP32 rate (and every FP32<->FP64
// conversion takes an FP64 issue slot), so arithmetic that needs more than FP32's 24 bits runs
// far faster as pairs of FP32 operations than as FP64.
//
// Every primitive rounds each operation separately (no contraction into fused multiply-adds
// except where written), which the error-free transformations require: on the device through
// the __f*_rn intrinsics, on the host (where this header is also compiled for tests) through
// plain FP32 expressions built with contraction disabled.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define LFX_HD __host__ __device__ __forceinline__
#else
#define LFX_HD inline
#endif

namespace lfx {

LFX_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
LFX_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
LFX_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
LFX_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}
LFX_HD float f_div(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}

struct dd {
  float hi, lo;
  dd() = default;
  LFX_HD constexpr dd(float h, float l) : hi(h), lo(l) {}
  // exact for small integers; a double is split into its nearest FP32 value and the remainder
  LFX_HD explicit dd(int v) : hi((float)v), lo(0.0f) {}
  LFX_HD explicit dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  LFX_HD explicit operator double() const { return (double)hi + (double)lo; }
  LFX_HD explicit operator float() const { return hi; }
};

// s + e = a + b exactly
LFX_HD dd two_sum(float a, float b) {
  const float s = f_add(a, b);
  const float v = f_sub(s, a);
  const float e = f_add(f_sub(a, f_sub(s, v)), f_sub(b, v));
  return dd(s, e);
}
// s + e = a + b exactly, given |a| >= |b| (or a == 0)
LFX_HD dd fast_two_sum(float a, float b) {
  const float s = f_add(a, b);
  return dd(s, f_sub(b, f_sub(s, a)));
}
// p + e = a * b exactly
LFX_HD dd two_prod(float a, float b) {
  const float p = f_mul(a, b);
  return dd(p, f_fma(a, b, -p));
}

LFX_HD dd operator-(dd a) { return dd(-a.hi, -a.lo); }

// sum with relative error O(2^-47) even under cancellation: the high parts and the low parts
// are each summed exactly, then renormalised.  Sums of contributions (matrix entries, element
// sums) use add_acc below instead, whose error bound is relative to the operands.
LFX_HD dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, f_add(s.lo, t.hi));
  return fast_two_sum(s.hi, f_add(s.lo, t.lo));
}
LFX_HD dd operator-(dd a, dd b) { return a + (-b); }

// a + b for accumulations: the high parts are summed exactly, the low parts and that sum's error
// in FP32, then renormalised (11 FP32 operations against 20).  The error is a few units of 2^-47
// of |a| + |b| (not of the result): the error model of recursive summation in a format with a
// 48-bit significand, which is what summing element contributions into a matrix entry needs.
LFX_HD dd add_acc(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, f_add(s.lo, f_add(a.lo, b.lo)));
}

LFX_HD dd operator*(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  float e = f_fma(a.hi, b.lo, p.lo);
  e = f_fma(a.lo, b.hi, e);
  return fast_two_sum(p.hi, e);
}

// quotient by long division: three FP32 quotient digits, each from the remainder so far
LFX_HD dd operator/(dd a, dd b) {
  const float q1 = f_div(a.hi, b.hi);
  dd r = a - b * dd(q1, 0.0f);
  const float q2 = f_div(r.hi, b.hi);
  r = r - b * dd(q2, 0.0f);
  const float q3 = f_div(r.hi, b.hi);
  const dd q = fast_two_sum(q1, q2);
  return q + dd(q3, 0.0f);
}

// a * b + c
LFX_HD dd fma_dd(dd a, dd b, dd c) { return a * b + c; }

// a * b + c in one pass: the product of the high parts and its sum with c.hi are exact (two_prod,
// two_sum); the cross products and every low-order part are summed in FP32, then renormalised.
// 15 FP32 operations against 27 for fma_dd.  The error is a few units of 2^-47 of
// max(|a b|, |c|) (not of the result: under cancellation the relative error of the result grows),
// which is the accuracy an accumulation of terms needs when its error is judged against the
// terms' own magnitude.
LFX_HD dd fma_dd_fast(dd a, dd b, dd c) {
  const dd p = two_prod(a.hi, b.hi);
  float e = f_fma(a.hi, b.lo, p.lo);
  e = f_fma(a.lo, b.hi, e);
  const dd s = two_sum(p.hi, c.hi);
  e = f_add(e, f_add(c.lo, s.lo));
  return fast_two_sum(s.hi, e);
}
LFX_HD dd &operator+=(dd &a, dd b) { return a = a + b; }
LFX_HD dd &operator-=(dd &a, dd b) { return a = a - b; }
LFX_HD dd &operator*=(dd &a, dd b) { return a = a * b; }

LFX_HD bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
LFX_HD bool operator>(dd a, dd b) { return b < a; }
LFX_HD bool operator==(dd a, dd b) { return a.hi == b.hi && a.lo == b.lo; }
LFX_HD bool operator!=(dd a, dd b) { return !(a == b); }
LFX_HD dd dd_abs(dd a) { return a.hi < 0.0f ? -a : a; }

// x^-1/2 for x > 0: FP32 estimate y0, then one Newton step y0 + y0 (1 - x y0^2) / 2 in dd (the
// step squares the estimate's relative error, about 2^-22 for the estimate, below dd rounding)
LFX_HD dd dd_rsqrt(dd x) {
#ifdef __CUDA_ARCH__
  const float y0 = rsqrtf(x.hi);
#else
  const float y0 = 1.0f / std::sqrt(x.hi);
#endif
  const dd y(y0, 0.0f);
  const dd h = dd(1.0f, 0.0f) - x * (y * y);
  return y + y * (h * dd(0.5f, 0.0f));
}

}  // namespace lfx
