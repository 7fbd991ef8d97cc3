// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// float32 numbers with |lo| <= ulp(hi)/2, about 48 bits of significand.
// Sums use Knuth's TwoSum (the exact error of a float32 addition) followed by
// Dekker's Fast2Sum renormalisation; products use the fused multiply-add for
// the exact error of hi*hi (the "TwoProduct" of Ogita, Rump and Oishi, 2005).
// Relative error of one operation about 2^-46 (sums of values of opposite
// signs lose no more than that of the larger operand).  Everything runs on
// the float32 pipes, which on this GPU have 64 times the float64 rate.
#pragma once

#include <cuda_runtime.h>

namespace cpc {

// A float32 as float64, exactly, by integer work on the IEEE-754 fields (the
// exponent rebiased from 127 to 1023, the mantissa moved to the top of the
// 52-bit field): no conversion instruction, which like the float64
// arithmetic runs at a small fraction of the float32 rate on this GPU.
// Subnormal floats (below 2^-126) are taken as zero.
__device__ __forceinline__ double double_of_float_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const unsigned long long ed = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | (ed << 52) |
                                          ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

struct __align__(8) df {
  float hi, lo;
  __host__ __device__ df() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
  // exact split of a double into its leading float and the rounded rest
  __host__ __device__ explicit df(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
  __host__ __device__ explicit df(int i) : df(double(i)) {}
  // hi + lo rounded to float64 (the conversion instructions: in the
  // double-float FFT, whose float32 pipes are the busy ones, they measured
  // faster than double_of_float_exact)
  __host__ __device__ double to_double() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ df df_fast2sum(float s, float e) {
  const float h = s + e;
  return df(h, e - (h - s));
}

__device__ __forceinline__ df operator+(df a, df b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  const float e = (a.hi - (s - v)) + (b.hi - v) + (a.lo + b.lo);
  return df_fast2sum(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return df_fast2sum(p, e);
}

// complex double-float (the FFT templates' V: members x, y)
struct __align__(16) dfc {
  df x, y;
};

}  // namespace cpc
