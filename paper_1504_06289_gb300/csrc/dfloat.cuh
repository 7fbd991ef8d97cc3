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

struct __align__(8) df {
  float hi, lo;
  __host__ __device__ df() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ df(float h, float l) : hi(h), lo(l) {}
  // exact split of a double into its leading float and the rounded rest
  __host__ __device__ explicit df(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
  __host__ __device__ explicit df(int i) : df(double(i)) {}
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
