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

}  // namespace fsib
