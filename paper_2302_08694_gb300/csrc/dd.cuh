// Double-float ("dd") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, about 48 significant bits. The error-free
// transformations are Knuth's TwoSum and the FMA-based TwoProd (Dekker's
// product with a fused multiply-add); the sums and products below follow the
// double-double algorithms of Hida, Li and Bailey (QD library paper, 2001),
// restated for float pairs. FP64 mode computes transforms in this type because
// GB300 executes FP32 arithmetic at a far higher rate than FP64 arithmetic.
//
// Every operation uses the _rn intrinsics so that no multiply and add pair is
// contracted into an FMA behind our back.
#pragma once
#include <cuda_runtime.h>
#include "ddconv.cuh"

namespace fsib {

struct __align__(8) dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dd(int x) : hi((float)x), lo(0.0f) {}
  __host__ __device__ constexpr dd(float x) : hi(x), lo(0.0f) {}
  // Exact split of a double into hi + lo (FP64 arithmetic: use at boundaries
  // and for compile-time constants only).
  __host__ __device__ constexpr dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

struct __align__(16) dd2 {  // 16-byte aligned so that a complex value moves as one vector
  dd x, y;
};

// double -> double-float on the integer and FP32 pipes (ddconv.cuh); magnitudes of 2^128 and
// above, infinities and NaN go through FP64.
__device__ __forceinline__ dd dd_from_double(double x) {
  float h, l;
  if (ddconv::split_double(x, h, l)) return dd(h, l);
  return dd(x);
}
// double-float -> double: both parts widened exactly by integer operations, then one FP64
// addition (a join of the pair by integer arithmetic alone measured slower than this form).
__device__ __forceinline__ double dd_to_double(dd v) {
  return ddconv::widen_float(v.hi) + ddconv::widen_float(v.lo);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Sum with one TwoSum on the high parts (norm-wise accurate, what FFT error analysis needs).
__device__ __forceinline__ dd operator+(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float h, l;
  quick_two_sum(s, e, h, l);
  return dd(h, l);
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float h, l;
  quick_two_sum(p, e, h, l);
  return dd(h, l);
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { a = a + b; return a; }

// Sum without the final renormalisation (8 instructions instead of 11): hi is the rounded sum
// of the high parts, lo the TwoSum error plus the low parts, so hi + lo is the same value as
// a + b above but |lo| may exceed ulp(hi)/2 by a few units. Chains of such sums (the butterflies
// of one DFT) keep their norm-wise error bound, which is what FFT error analysis needs; a
// later product or renormalising sum restores the canonical form.
__device__ __forceinline__ dd dd_add_nr(dd a, dd b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return dd(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

// a b + c d with one TwoSum: each product formed by TwoProd plus its two cross terms, the
// high parts added by TwoSum, every error term by plain adds, one renormalisation at the end
// (19 instructions instead of 25 for two rounded products and a sum).
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d) {
  float p, e, q, f;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  two_prod(c.hi, d.hi, q, f);
  f = __fmaf_rn(c.hi, d.lo, f);
  f = __fmaf_rn(c.lo, d.hi, f);
  float s, r;
  two_sum(p, q, s, r);
  r = __fadd_rn(r, __fadd_rn(e, f));
  float h, l;
  quick_two_sum(s, r, h, l);
  return dd(h, l);
}

// Exact halving (a power-of-two scale of both parts).
__device__ __forceinline__ dd dd_half(dd a) { return dd(__fmul_rn(0.5f, a.hi), __fmul_rn(0.5f, a.lo)); }

// Accumulator for long sums of products: acc.hi collects the rounded sum, acc.lo the
// exact rounding errors (TwoSum) plus the low parts; renormalised only when read.
// The product a*b is formed without the final renormalisation (TwoProd plus the two
// cross terms), which is enough when it only feeds an accumulator.
__device__ __forceinline__ void dd_fma_acc(dd& acc, dd a, dd b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, r;
  two_sum(acc.hi, p, s, r);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(r, e));
}
__device__ __forceinline__ dd dd_norm(dd a) {
  float h, l;
  quick_two_sum(a.hi, a.lo, h, l);
  return dd(h, l);
}
__device__ __forceinline__ dd& operator*=(dd& a, dd b) { a = a * b; return a; }

// Square root of a non-negative value: one Newton correction of the FP32 root,
// r + (a - r^2) / (2 r), with r^2 formed exactly by TwoProd (Karp and Markstein's form).
__device__ __forceinline__ dd dd_sqrt(dd a) {
  if (!(a.hi > 0.0f)) return dd(0.0f, 0.0f);
  const float r = __fsqrt_rn(a.hi);
  float p, e;
  two_prod(r, r, p, e);
  const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);  // a.hi - p is exact
  const float c = __fmul_rn(res, __fdiv_rn(0.5f, r));
  float h, l;
  quick_two_sum(r, c, h, l);
  return dd(h, l);
}

// exp(y) for -60 <= y <= 0 (the kernel's exponent). Range reduction y = k ln2 + t with
// |t| <= ln2/2, ln2 split into three floats so that t is formed almost exactly (Cody and
// Waite); e^t by its Taylor series to degree 14 (remainder below 1e-19) evaluated by
// Horner's rule in double-float; the result is scaled by 2^k.
__device__ __forceinline__ dd dd_exp_nonpos(dd y) {
  const float k = rintf(__fmul_rn(y.hi, 1.4426950408889634f));
  const float L1 = 0.693359375f, L2 = -2.1219444170128554e-4f, L3 = 1.6465949697480609e-12f;
  const float a = __fsub_rn(y.hi, __fmul_rn(k, L1));  // exact: k L1 has at most 17 bits
  float p2, e2;
  two_prod(k, L2, p2, e2);
  float s, se;
  two_sum(a, -p2, s, se);
  const float small = __fadd_rn(__fadd_rn(__fsub_rn(se, e2), -__fmul_rn(k, L3)), y.lo);
  float th, tl;
  quick_two_sum(s, small, th, tl);
  const dd t(th, tl);
  // 1/n! for n = 14 .. 0
  constexpr dd c14(1.0 / 87178291200.0), c13(1.0 / 6227020800.0), c12(1.0 / 479001600.0),
      c11(1.0 / 39916800.0), c10(1.0 / 3628800.0), c9(1.0 / 362880.0), c8(1.0 / 40320.0),
      c7(1.0 / 5040.0), c6(1.0 / 720.0), c5(1.0 / 120.0), c4(1.0 / 24.0), c3(1.0 / 6.0), c2(0.5),
      c1(1.0), c0(1.0);
  dd P = c14;
  P = P * t + c13; P = P * t + c12; P = P * t + c11; P = P * t + c10; P = P * t + c9;
  P = P * t + c8;  P = P * t + c7;  P = P * t + c6;  P = P * t + c5;  P = P * t + c4;
  P = P * t + c3;  P = P * t + c2;  P = P * t + c1;  P = P * t + c0;
  const float sc = __int_as_float((127 + (int)k) << 23);  // 2^k, exact (k >= -87)
  return dd(__fmul_rn(P.hi, sc), __fmul_rn(P.lo, sc));
}

}  // namespace fsib
