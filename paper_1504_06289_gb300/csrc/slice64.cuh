// The five weighted bf16 digits of a float64 value for the float64-accurate
// tensor-core contraction (CPC_FP64_TC): x = 2^(e-8) sum_j t_j with
// t_j = s_j 2^(-8j), |s_0| <= 256, |s_j| <= 128, taken from the integer bit
// pattern of x (one round-to-nearest shift to the row's 2^(e-40) grid, then
// 8-bit fields with a bias of 128 per byte), exact and free of float64
// arithmetic.  e is the row exponent: 2^e > max |x| over the row, here the
// largest biased exponent field of the row minus 1022 (0 for a row of zeros);
// a larger e is valid too and keeps fewer of the value's bits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace cpc {

constexpr int kSlice64 = 5;   // digits per value
constexpr int kSlice64Cells = 32;  // cells per chunk of the slice layout

// Integer to float without a conversion instruction: for 0 <= v < 2^23 the
// bit pattern 0x4B000000 | v is the float 2^23 + v, and (2^23 + v) w - c w,
// with c = 2^23 plus the digit's bias and w its weight (a signed power of
// two), is one exact fused multiply-add (the result is a float).
__device__ __forceinline__ void slice64_digits(double x, int e, float t[kSlice64]) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int ex = int((bits >> 52) & 0x7FF);
  const int sh = 1035 + e - ex;
  long long A = 0;
  if (ex != 0 && sh < 64) {
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    A = (long long)((mant + (1ull << (sh - 1))) >> sh);
  }
  const unsigned sbit = unsigned(bits >> 63) << 31;
  const unsigned long long B = (unsigned long long)A + 0x80808080ull;
  const unsigned hi = unsigned(B >> 32), lo = unsigned(B);
  // leading digit hi in [0, 256], weight +-1
  const float w0 = __uint_as_float(0x3F800000u | sbit);
  t[0] = fmaf(__uint_as_float(0x4B000000u | hi), w0, -8388608.0f * w0);
#pragma unroll
  for (int j = 1; j < kSlice64; ++j) {
    // byte 4 - j of lo, biased by 128, weight +-2^(-8j)
    const float w = __uint_as_float((unsigned(127 - 8 * j) << 23) | sbit);
    const float f = __uint_as_float(__byte_perm(lo, 0x4B000000u, unsigned(kSlice64 - 1 - j) | 0x7650u));
    t[j] = fmaf(f, w, -8388736.0f * w);  // (2^23 + b) w - (2^23 + 128) w = (b - 128) w
  }
}

// the biased exponent field of x (0 for zeros and subnormals)
__device__ __forceinline__ int biased_exponent64(double x) {
  return int((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7FF);
}
// row exponent from the largest biased exponent field of the row
__device__ __forceinline__ int row_exponent64(int max_biased) { return max_biased ? max_biased - 1022 : 0; }

// the digits of the outputs x0, x1 (cells i, i+1 of one 32-cell chunk) stored
// as bf16 pairs at o + j stride, j < 5 (streaming stores: the slices are
// read once, by the contraction, and must not push its operands out of L2)
__device__ __forceinline__ void slice64_pair(double x0, double x1, int e, __nv_bfloat16* o, long long stride) {
  float t0[kSlice64], t1[kSlice64];
  slice64_digits(x0, e, t0);
  slice64_digits(x1, e, t1);
  // every digit has at most 8 significant bits: its bf16 is the top half of
  // its float (cell i in the low half)
#pragma unroll
  for (int j = 0; j < kSlice64; ++j)
    __stcs(reinterpret_cast<unsigned int*>(o + j * stride),
           __byte_perm(__float_as_uint(t0[j]), __float_as_uint(t1[j]), 0x7632u));
}

}  // namespace cpc
