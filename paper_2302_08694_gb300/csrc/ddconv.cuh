// Conversions between double and the double-float pair (hi, lo) without FP64 conversions.
// GB300 runs FP64 instructions, conversions to and from FP64 included, at a small fraction of
// its FP32 rate, so a pass that reads or writes FP64 spectra spent most of its FP64-pipe time
// converting. The split takes the IEEE-754 fields of the double apart with integer operations
// (the remainder's 29 bits go through one integer-to-float conversion); the widening of a
// float is pure bit arithmetic. Magnitudes of 2^128 and above, infinities and NaN take the
// FP64 path (the caller's fallback).
//
// Plain C++ on both sides (host and device), so the host build can be checked against exact
// rational arithmetic.
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#endif

namespace fsib {
namespace ddconv {

__host__ __device__ inline uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
#endif
}
__host__ __device__ inline float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, 4);
  return f;
#endif
}
__host__ __device__ inline uint64_t d2u(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  std::memcpy(&u, &d, 8);
  return u;
#endif
}
__host__ __device__ inline double u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  std::memcpy(&d, &u, 8);
  return d;
#endif
}
__host__ __device__ inline float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

// An unsigned integer as a float, rounded to nearest (an I2F, which measured cheaper than
// building the float from two exact halves).
__host__ __device__ inline float uint_to_float_rn(uint32_t r) {
#ifdef __CUDA_ARCH__
  return __uint2float_rn(r);
#else
  return (float)r;
#endif
}

// x = hi + lo with hi the significand of x cut to 24 bits (towards zero) and lo the remaining 29
// bits rounded to 24, so |lo| <= ulp(hi) and |x - (hi + lo)| <= 2^-48 |x|, for 2^-74 <= |x| <
// 2^128. Below 2^-74 lo would leave FP32's normal range: there lo = 0 (an error under 2^-97),
// and below 2^-126 also hi = 0 (zero and denormal doubles included), both with x's sign.
// Returns false (and leaves hi, lo alone) for |x| >= 2^128, infinities and NaN.
__host__ __device__ inline bool split_double(double x, float& hi, float& lo) {
  const uint64_t b = d2u(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const int e = (int)((hw >> 20) & 0x7FFu);  // biased exponent
  if (e > 1150) return false;
  const uint32_t sign = hw & 0x80000000u;
  if (e < 897) {  // |x| < 2^-126
    hi = u2f(sign);
    lo = u2f(sign);
    return true;
  }
  hi = u2f(sign | ((uint32_t)(e - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  if (e < 949) {  // the remainder's scale 2^(e - 1075) would not be a normal float
    lo = u2f(sign);
    return true;
  }
  const uint32_t r = lw & 0x1FFFFFFFu;                    // remainder, 29 bits
  const float s = u2f((uint32_t)(e - 1075 + 127) << 23);  // 2^(e - 1075)
  const float mag = mul_rn(uint_to_float_rn(r), s);       // r rounded to 24 bits, scaled exactly
  lo = sign ? -mag : mag;
  return true;
}

// A float as a double, exactly, by integer operations: zero and denormals (below 2^-126) give a
// signed zero; infinities and NaN are converted in FP64.
__host__ __device__ inline double widen_float(float f) {
  const uint32_t b = f2u(f);
  const uint32_t ex = (b >> 23) & 0xFFu;
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  if (ex == 0) return u2d(sign);
  if (ex == 255) return (double)f;
  return u2d(sign | ((uint64_t)(ex - 127 + 1023) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29));
}

}  // namespace ddconv
}  // namespace fsib
