// Batched 1D convolutions of CP factors with the Newton-kernel vectors
// (Sec. 2.5, Eq. conv; the V_H factors of Sec. 3.1) by length-2n real FFTs.
//
// Each column is zero-padded to 2n real points; a length-2n real transform is
// an n-point complex transform of the packed pairs (x[2j], x[2j+1]) plus a
// half-angle post/pre-processing step.  The linear convolution with a kernel
// given on offsets -(n-1)..n-1 is exact on outputs 0..n-1 under the 2n
// circular convolution (the wrap-around lands on outputs n..2n-1, which are
// never formed).
//
//   spectra_kernel : float64 forward transforms of factor columns (and of the
//                    kernel vectors at set-up), stored as n+1 Hermitian bins.
//   conv_kernel    : per (column, q) item, multiply by the kernel spectrum,
//                    inverse transform, keep the first n outputs.  One CTA
//                    holds `slots` transforms in shared memory and walks the
//                    items in a grid-stride loop.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "cpc_internal.h"
#include "fft.cuh"
#include "slice64.cuh"

namespace cpc {

namespace {

constexpr int kMaxLogN = 13;  // n <= 8192 for convolution kernels
constexpr int kMinLogN = 4;

// points per thread: 16 (float64, small n) or 32 (float32, n >= 1024: three passes for n = 8192)
template <typename T, int LOGN> constexpr int pick_logp() {
  return LOGN <= 4 ? LOGN - 1 : ((sizeof(T) == 4 && LOGN >= 10) ? 5 : 4);
}

template <int LOGN, typename T = double>
struct Geometry {
  static constexpr int LOGP = pick_logp<T, LOGN>();
  using PL = FftPlan<LOGN, LOGP>;
  static constexpr int slots = PL::TPF >= 256 ? 1 : 256 / PL::TPF;
  static constexpr int threads = slots * PL::TPF;
  static constexpr int min_blocks = threads >= 512 ? 1 : 2;
};

// ---------------------------------------------------------------------------
// forward spectra (float64).  mode 0: factor columns (zero padded to 2n);
// mode 1: even kernel vectors p[0..n-1] extended to the 2n circle;
// mode 2: factor columns, written as the float32 convolution operands
//   X1[f] = U^[f] (1 + i e^{i theta_f}),  X2[f] = conj(U^[n-f]) (1 - i e^{i theta_f}),
//   theta_f = pi f / n, f = 0..n-1 (out4[col][f] = (X1, X2)), so that the
//   convolution's packed spectrum is Z[f] = p^[f] X1[f] + p^[n-f] X2[f].
template <int LOGN>
__global__ void __launch_bounds__(Geometry<LOGN>::threads)
spectra_kernel(int mode, const double* __restrict__ src, int ncols, double2* __restrict__ out64,
               float2* __restrict__ out32, double* __restrict__ re64, float* __restrict__ re32,
               const double2* __restrict__ hw, const double2* __restrict__ tw, float4* __restrict__ out4) {
  using G = Geometry<LOGN>;
  using PL = typename G::PL;
  constexpr int NC = PL::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* sbuf = reinterpret_cast<double2*>(smem_raw) + (threadIdx.x / PL::TPF) * padded_len(NC);
  const int slot = threadIdx.x / PL::TPF;
  const int t = threadIdx.x % PL::TPF;
  for (int g = blockIdx.x; g * G::slots < ncols; g += gridDim.x) {
    const int col = g * G::slots + slot;
    const bool active = col < ncols;
    const double* x = src + (size_t)(active ? col : ncols - 1) * NC;
    {
      double2 v[PL::B1][PL::R1];
      constexpr int stride = NC / PL::R1, nbf = NC / (PL::R1 * PL::B1);
#pragma unroll
      for (int b = 0; b < PL::B1; ++b) {
        const int j = b * nbf + t;
#pragma unroll
        for (int r = 0; r < PL::R1; ++r) {
          const int f = j + r * stride;  // packed pair (x[2f], x[2f+1])
          double2 z;
          if (mode != 1) {
            z = (2 * f < NC) ? *reinterpret_cast<const double2*>(x + 2 * f) : make_double2(0.0, 0.0);
          } else {
            const int m0 = 2 * f, m1 = 2 * f + 1;
            const double a0 = m0 < NC ? x[m0] : (m0 == NC ? 0.0 : x[2 * NC - m0]);
            const double a1 = m1 < NC ? x[m1] : x[2 * NC - m1];
            z = make_double2(a0, a1);
          }
          v[b][r] = z;
        }
        dft<PL::R1, -1>(v[b]);
      }
      pass_store<NC, PL::R1, PL::B1>(sbuf, v, t, 1);
    }
    __syncthreads();
    middle_passes<LOGN, G::LOGP, -1>(sbuf, t, tw, nullptr);
    {
      double2 v[1][PL::P];
      pass_compute<NC, PL::P, 1, -1>(sbuf, v, t, NC / PL::P, tw + pass_table_offset<LOGN, G::LOGP>(PL::NP - 1),
                                     nullptr);
      __syncthreads();
      pass_store<NC, PL::P, 1>(sbuf, v, t, NC / PL::P);
    }
    __syncthreads();
    // X[f] = (Z[f] + conj Z[n-f])/2 - (i/2) e^{-2 pi i f/2n} (Z[f] - conj Z[n-f]), f = 0..n
    auto bin = [&](int f) {
      const double2 Zf = sbuf[pad_index(f & (NC - 1))];
      const double2 Zr = cconj(sbuf[pad_index((NC - f) & (NC - 1))]);
      const double2 s = cadd(Zf, Zr), d = csub(Zf, Zr);
      const double2 wd = cmul(hw[f], d);  // e^{-i theta} (Z - conj Z')
      return make_double2(0.5 * s.x + 0.5 * wd.y, 0.5 * s.y - 0.5 * wd.x);
    };
    if (active && mode == 2) {
      // bins f and n-f give the operands at both f and n-f: one pair per step
      auto operands = [&](int f, double2 Uf, double2 Un) {  // Un = U^[n-f]
        const double2 E = cconj(hw[f]);             // e^{+i theta_f}
        const double2 iE = make_double2(-E.y, E.x);  // i e^{+i theta_f}
        const double2 X1 = cmul(Uf, make_double2(1.0 + iE.x, iE.y));
        const double2 X2 = cmul(cconj(Un), make_double2(1.0 - iE.x, -iE.y));
        out4[(size_t)col * NC + f] = make_float4(float(X1.x), float(X1.y), float(X2.x), float(X2.y));
      };
      for (int f = t; f <= NC / 2; f += PL::TPF) {
        const double2 Uf = bin(f), Un = bin(NC - f);
        operands(f, Uf, Un);
        if (f > 0 && 2 * f < NC) operands(NC - f, Un, Uf);
      }
    } else if (active) {
      for (int f = t; f <= NC; f += PL::TPF) {
        const double2 Zf = sbuf[pad_index(f & (NC - 1))];
        const double2 Zr = cconj(sbuf[pad_index((NC - f) & (NC - 1))]);
        const double2 s = cadd(Zf, Zr), d = csub(Zf, Zr);
        const double2 w = hw[f];
        const double2 wd = cmul(w, d);  // e^{-i theta} (Z - conj Z')
        // -(i/2) * wd = (wd.y/2, -wd.x/2)
        const double2 X = make_double2(0.5 * s.x + 0.5 * wd.y, 0.5 * s.y - 0.5 * wd.x);
        const size_t o = (size_t)col * (NC + 1) + f;
        if (mode == 0) {
          if (out64) out64[o] = X;
          if (out32) out32[o] = make_float2(float(X.x), float(X.y));
        } else {
          if (re64) re64[o] = X.x;
          if (re32) re32[o] = float(X.x);
        }
      }
    }
    __syncthreads();
  }
}

// Float32 forward transform for the float32 form's convolution operands
// (the output of spectra_kernel mode 2), with the float32 plan and the
// compensated constants and twiddles of fft.cuh; inputs rounded to float32
// once; the operand factors (1 +- i e^{i theta}) formed in float64.
template <int LOGN>
__global__ void __launch_bounds__(Geometry<LOGN, float>::threads)
spectra32_kernel(const double* __restrict__ src, int ncols, const float2* __restrict__ hw,
                 const __half2* __restrict__ hwl, const float4* __restrict__ opf, const float2* __restrict__ tw,
                 const __half2* __restrict__ twl, float4* __restrict__ out4) {
  using G = Geometry<LOGN, float>;
  using PL = typename G::PL;
  constexpr int NC = PL::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* sbuf = reinterpret_cast<float2*>(smem_raw) + (threadIdx.x / PL::TPF) * padded_len(NC);
  const int slot = threadIdx.x / PL::TPF;
  const int t = threadIdx.x % PL::TPF;
  for (int g = blockIdx.x; g * G::slots < ncols; g += gridDim.x) {
    const int col = g * G::slots + slot;
    const bool active = col < ncols;
    const double* x = src + (size_t)(active ? col : ncols - 1) * NC;
    {
      float2 v[PL::B1][PL::R1];
      constexpr int stride = NC / PL::R1, nbf = NC / (PL::R1 * PL::B1);
#pragma unroll
      for (int b = 0; b < PL::B1; ++b) {
        const int j = b * nbf + t;
#pragma unroll
        for (int r = 0; r < PL::R1; ++r) {
          const int f = j + r * stride;  // packed pair (x[2f], x[2f+1]), zero beyond n
          if (2 * f < NC) {
            const double2 z = *reinterpret_cast<const double2*>(x + 2 * f);
            v[b][r] = make_float2(float(z.x), float(z.y));
          } else {
            v[b][r] = make_float2(0.0f, 0.0f);
          }
        }
        dft<PL::R1, -1>(v[b]);
      }
      pass_store<NC, PL::R1, PL::B1>(sbuf, v, t, 1);
    }
    __syncthreads();
    middle_passes<LOGN, G::LOGP, -1>(sbuf, t, tw, twl);
    {
      float2 v[1][PL::P];
      constexpr int off = pass_table_offset<LOGN, G::LOGP>(PL::NP - 1);
      pass_compute<NC, PL::P, 1, -1>(sbuf, v, t, NC / PL::P, tw + off, twl + off);
      __syncthreads();
      pass_store<NC, PL::P, 1>(sbuf, v, t, NC / PL::P);
    }
    __syncthreads();
    if (active) {
      // U^[f] = (Z[f] + conj Z[n-f])/2 - (i/2) e^{-i theta} (Z[f] - conj Z[n-f])
      auto bin = [&](int f) {
        const float2 Zf = sbuf[pad_index(f & (NC - 1))];
        const float2 Zr = cconj(sbuf[pad_index((NC - f) & (NC - 1))]);
        const float2 sm = cadd(Zf, Zr), d = csub(Zf, Zr);
        const float2 wd = twiddle<-1>(d, hw, hwl, f);  // e^{-i theta} (Z - conj Z'), compensated
        return make_float2(0.5f * sm.x + 0.5f * wd.y, 0.5f * sm.y - 0.5f * wd.x);
      };
      auto operands = [&](int f, float2 Uf, float2 Un) {  // Un = U^[n-f]
        // (1 + i e^{+i theta}, 1 - i e^{+i theta}) formed in float64 and rounded
        // once, from the table built with the kernel (operand_factor_kernel)
        const float4 a = __ldg(opf + f);
        const float2 a1 = make_float2(a.x, a.y), a2 = make_float2(a.z, a.w);
        const float2 X1 = cmul(Uf, a1), X2 = cmul(cconj(Un), a2);
        out4[(size_t)col * NC + f] = make_float4(X1.x, X1.y, X2.x, X2.y);
      };
      for (int f = t; f <= NC / 2; f += PL::TPF) {
        const float2 Uf = bin(f), Un = bin(NC - f);
        operands(f, Uf, Un);
        if (f > 0 && 2 * f < NC) operands(NC - f, Un, Uf);
      }
    }
    __syncthreads();
  }
}

// Optional second output of the convolution: the exact bf16 slices of each
// output row (the operand format of the tensor-core contraction,
// csrc/gram_tc.cu), written in the chunk-blocked layout (SliceRows) and with
// the same arithmetic as slice_rows_kernel (float32 W) or slice64_kernel
// (float64 W), so the result is bit-identical where the row exponent is the
// same.
using SliceOut = SliceRows;

// 2^(8-e) as two normal powers of two (here e is in [-147, 129]): two exact
// multiplies per value instead of ldexpf (a value whose first product would
// fall below the normal range is below the last digit)
__device__ __forceinline__ void slice_scales(int e, float& sc1, float& sc2) {
  const int k1 = (8 - e) / 2, k2 = (8 - e) - k1;
  sc1 = __int_as_float((127 + k1) << 23);
  sc2 = __int_as_float((127 + k2) << 23);
}

// the three balanced digits of the outputs x0, x1 (cells i, i+1 of one
// 64-cell chunk) under the row scale, stored as bf16 pairs at o, o + stride,
// o + 2 stride with streaming stores (evict first: the outputs must not push
// the reused operands out of L2)
__device__ __forceinline__ void slice_pair(float x0, float x1, float sc1, float sc2, __nv_bfloat16* o,
                                           long long stride) {
  float sl[3][2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const float a = ((h ? x1 : x0) * sc1) * sc2;  // |a| < 128
    const float s0 = rintf(a);
    const float b = (a - s0) * 256.0f;  // exact
    const float s1 = rintf(b);
    sl[0][h] = s0;
    sl[1][h] = s1;
    sl[2][h] = rintf((b - s1) * 256.0f);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(sl[k][0], sl[k][1]);
    __stcs(reinterpret_cast<unsigned int*>(o + k * stride), *reinterpret_cast<const unsigned int*>(&b2));
  }
}

// balanced-digit row exponent of the float32 form's W operand: 2^e > 2 max|x|
__device__ __forceinline__ int balanced_exponent(float m) {
  int e = 0;
  if (m > 0.0f) {
    frexpf(m, &e);
    e += 1;
  }
  return e;
}

// Row maximum over the TPF threads of one transform, then the three slices of
// each of this thread's outputs (reals 2o, 2o+1, o = t + r NC/P, r < P/2).
template <typename PL>
__device__ __forceinline__ void slice_epilogue(const float2* v, const SliceOut& so, long long item, bool active,
                                               int slot, int t, int R_N) {
  constexpr int NC = PL::NC, TPF = PL::TPF;
  __shared__ float red[32];  // per-warp maxima (transforms of >= 32 threads)
  float m = 0.0f;
#pragma unroll
  for (int r = 0; r < PL::P / 2; ++r) m = fmaxf(m, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
  // within a warp: lanes of the same transform (TPF lanes, or all 32)
  constexpr int LW = TPF < 32 ? TPF : 32;
#pragma unroll
  for (int o = LW / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if constexpr (TPF > 32) {
    // a transform spans TPF / 32 whole warps: combine them
    constexpr int WPF = TPF / 32;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = red[slot * WPF];
#pragma unroll
    for (int w = 1; w < WPF; ++w) m = fmaxf(m, red[slot * WPF + w]);
    __syncthreads();  // red[] is reused by the next item
  }
  if (!active) return;
  const int e = balanced_exponent(m);
  if (t == 0) so.expo[item] = e;
  const long long col = item / R_N;
  const int q = int(item - col * R_N);
  const int l = int(col / so.R_f), srow = int(col - (long long)l * so.R_f);
  constexpr int T = NC / 64;
  __nv_bfloat16* ob = so.out + ((long long)(l * R_N + q) * T * so.R_f + srow) * 64;
  float sc1, sc2;
  slice_scales(e, sc1, sc2);
#pragma unroll
  for (int r = 0; r < PL::P / 2; ++r) {
    const int i = 2 * (t + r * (NC / PL::P));  // even: the pair (i, i+1) stays in one 64-cell chunk
    slice_pair(v[r].x, v[r].y, sc1, sc2, ob + (long long)(i >> 6) * so.R_f * 64 + (i & 63), so.slice_stride);
  }
}

// The float64 counterpart (double-float transforms of CPC_FP64_TC): the row's
// largest biased exponent field over the TPF threads of one transform (from
// the values in registers), then the five digits of each of this thread's
// outputs (reals 2o, 2o+1) in the 32-cell chunks of the float64 form.  The
// digits are taken in a loop that is not unrolled, from the values staged in
// the transform's own shared buffer `sb` (free once every thread has passed
// the barrier at entry): unrolled over the outputs, the digit code overflows
// the instruction cache of the (fully unrolled) transform.
template <typename PL>
__device__ __forceinline__ void slice64_epilogue(const double2* v, double2* sb, const SliceOut& so, long long item,
                                                 bool active, int slot, int t, int R_N) {
  constexpr int NC = PL::NC, TPF = PL::TPF, C = kSlice64Cells;
  __shared__ int red64[32];
  int m = 0;
#pragma unroll
  for (int r = 0; r < PL::P / 2; ++r) m = max(m, max(biased_exponent64(v[r].x), biased_exponent64(v[r].y)));
  constexpr int LW = TPF < 32 ? TPF : 32;
#pragma unroll
  for (int o = LW / 2; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();  // every thread's last reads of the transform buffer are done
#pragma unroll
  for (int r = 0; r < PL::P / 2; ++r) sb[t + r * (NC / PL::P)] = v[r];
  if constexpr (TPF > 32) {
    constexpr int WPF = TPF / 32;
    if ((threadIdx.x & 31) == 0) red64[threadIdx.x >> 5] = m;
    __syncthreads();
    m = red64[slot * WPF];
#pragma unroll
    for (int w = 1; w < WPF; ++w) m = max(m, red64[slot * WPF + w]);
    __syncthreads();
  }
  if (!active) return;
  const int e = row_exponent64(m);
  if (t == 0) so.expo[item] = e;
  const long long col = item / R_N;
  const int q = int(item - col * R_N);
  const int l = int(col / so.R_f), srow = int(col - (long long)l * so.R_f);
  __nv_bfloat16* ob = so.out + ((long long)(l * R_N + q) * (NC / C) * so.R_f + srow) * C;
#pragma unroll 1
  for (int r = 0; r < PL::P / 2; ++r) {
    const int o = t + r * (NC / PL::P), i = 2 * o;
    const double2 x = sb[o];  // this thread's own entry
    slice64_pair(x.x, x.y, e, ob + (long long)(i / C) * so.R_f * C + (i % C), so.slice_stride);
  }
}

// ---------------------------------------------------------------------------
// batched convolution: item = col * R_N + q writes W[item][0..n-1].
// loads that ask L2 to keep the line (the convolution operands are read once
// per kernel term while the output stream passes through L2)
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_keep4(const float4* a, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;\n"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ float2 ld_keep2(const float2* a, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;\n" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
  return v;
}

// XIN: the factor spectra come as the float32 operands (X1, X2) of
// spectra_kernel mode 2 (`Uhat` points at float4 [cols][n]) and `phat` at
// the kernel-term pairs (p^[f], p^[n-f]) as float2 [R_N][n]; the packed
// spectrum is then Z[f] = p^[f] X1[f] + p^[n-f] X2[f] (no half-angle step).
// The kernel terms it convolves: qlist[0..n_q) (NULL: all R_N terms).  A
// group is one term for `slots` consecutive columns, so every transform of a
// CTA takes the same path and the same barriers.
template <typename T, int LOGN, bool SLICE, bool XIN = false>
__global__ void __launch_bounds__(Geometry<LOGN, T>::threads, Geometry<LOGN, T>::min_blocks)
conv_kernel(const typename cvec<T>::type* __restrict__ Uhat, const T* __restrict__ phat,
            const typename cvec<T>::type* __restrict__ hw, const typename cvec<T>::type* __restrict__ tw,
            const __half2* __restrict__ hwl, const __half2* __restrict__ twl,
            T* __restrict__ W, int R_N, int ncols, const int* __restrict__ qlist, int n_q, SliceOut so) {
  using V = typename cvec<T>::type;
  using G = Geometry<LOGN, T>;
  using PL = typename G::PL;
  constexpr int NC = PL::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = threadIdx.x / PL::TPF;
  const int t = threadIdx.x % PL::TPF;
  V* sbuf = reinterpret_cast<V*>(smem_raw) + slot * padded_len(NC);
  const T scale = T(1) / T(2 * NC);
  const uint64_t keep = l2_evict_last();  // operands are reused by the R_N kernel terms of a column
  // contiguous group range per CTA: consecutive groups share the factor
  // columns, so their spectra stay in L1 across the kernel terms q
  const long long n_groups = (long long)((ncols + G::slots - 1) / G::slots) * n_q;
  const long long g_begin = n_groups * blockIdx.x / gridDim.x;
  const long long g_end = n_groups * (blockIdx.x + 1) / gridDim.x;
  for (long long g = g_begin; g < g_end; ++g) {
    const long long cb = g / n_q;
    const int qi = int(g - cb * n_q);
    const int q = qlist ? __ldg(qlist + qi) : qi;
    const long long colr = cb * G::slots + slot;
    const bool active = colr < ncols;
    const long long col = active ? colr : ncols - 1;
    const long long item = col * R_N + q;
    const V* Uc = Uhat + (size_t)col * (NC + 1);
    const T* pq = phat + (size_t)q * (NC + 1);
    {
      // Z'[f] = (A + B) + i e^{+2 pi i f/2n} (A - B), A = Y[f], B = conj Y[n-f], Y = Uhat * phat
      V v[PL::B1][PL::R1];
      constexpr int stride = NC / PL::R1, nbf = NC / (PL::R1 * PL::B1);
#pragma unroll
      for (int b = 0; b < PL::B1; ++b) {
        const int j = b * nbf + t;
#pragma unroll
        for (int r = 0; r < PL::R1; ++r) {
          const int f = j + r * stride;
          if constexpr (XIN) {
            const float4 x = ld_keep4(reinterpret_cast<const float4*>(Uhat) + (size_t)col * NC + f, keep);
            const float2 pp = ld_keep2(reinterpret_cast<const float2*>(phat) + (size_t)q * NC + f, keep);
            v[b][r] = cmk<V>(fmaf(pp.x, x.x, pp.y * x.z), fmaf(pp.x, x.y, pp.y * x.w));
            continue;
          }
          const V uf = __ldg(Uc + f), ur = __ldg(Uc + (NC - f));
          const T pf = __ldg(pq + f), pr = __ldg(pq + (NC - f));
          const V A = cmk<V>(uf.x * pf, uf.y * pf);
          const V B = cmk<V>(ur.x * pr, -ur.y * pr);
          const V s = cadd(A, B), d = csub(A, B);
          const V wd = twiddle<+1>(d, hw, hwl, f);  // e^{+i theta} (A - B)
          v[b][r] = cmk<V>(s.x - wd.y, s.y + wd.x);
        }
        dft<PL::R1, +1>(v[b]);
      }
      pass_store<NC, PL::R1, PL::B1>(sbuf, v, t, 1);
    }
    __syncthreads();
    middle_passes<LOGN, G::LOGP, +1>(sbuf, t, tw, twl);
    {
      V v[1][PL::P];
      pass_compute<NC, PL::P, 1, +1>(sbuf, v, t, NC / PL::P, tw + pass_table_offset<LOGN, G::LOGP>(PL::NP - 1),
                                     twl ? twl + pass_table_offset<LOGN, G::LOGP>(PL::NP - 1) : nullptr);
#pragma unroll
      for (int r = 0; r < PL::P / 2; ++r) v[0][r] = cmk<V>(v[0][r].x * scale, v[0][r].y * scale);
      if (active) {
        T* out = W + (size_t)item * NC;
#pragma unroll
        for (int r = 0; r < PL::P / 2; ++r) {
          const int o = t + r * (NC / PL::P);  // complex output o -> reals 2o, 2o+1
          __stcs(reinterpret_cast<V*>(out + 2 * o), v[0][r]);  // streaming store (see slice_epilogue)
        }
      }
      if constexpr (SLICE) slice_epilogue<PL>(v[0], so, item, active, slot, t, R_N);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Banded direct convolution of the narrow kernel terms (Sec. 2.5, Eq. conv,
// as the finite sum it is).  The Galerkin vector p_q of a term with a large
// exponent t_q is a bell a few cells wide: beyond a half-width H_q its
// entries add up to less than a set fraction of sum_m |p_q[|m|]| (2^-32 for
// float32 W, 2^-60 for float64 W; build_term_tables picks H_q from the host
// float64 tables), and
//   W[i] = sum_{|m| <= H} p_q[|m|] U[i - m]      (U = 0 outside the grid)
// costs about 2H + 1 multiply-adds per output instead of a length-2n
// transform.  float32: each tap is a pair (hi, lo), lo the rounding error of
// hi; the lo products are kept for |m| <= (H+1)/2 (the host widens H until
// the taps beyond that add up to less than 2^-9 of the sum, so the dropped lo
// products stay below 2^-33 of it), so the rounding of the taps leaves no
// bias that would repeat across the columns of a term.  One CTA walks a
// contiguous range of (column, term) items, stages each column once in
// shared memory (rounded to T, as the FFT path rounds its input, inside a
// zero border of kBandHalo cells) and writes W, and with SLICE the bf16
// slices and row exponent: float32 W with the FFT path's arithmetic (row
// maximum over the CTA); float64 W with the row exponent bounded from the
// taps and the column (BandSlice64), so the digits are written as computed.
constexpr int kBandHalo = 32;          // largest half-width and the zero border
constexpr int kBandTaps = kBandHalo + 1;
constexpr int kBandThreads = 256;
// the half-widths with a kernel instantiation (a term's H is rounded up to one)
constexpr int kBandNumWidths = 17;
__host__ __device__ constexpr int band_width(int k) {
  return k < 9 ? k : (k < 13 ? 10 + 2 * (k - 9) : 20 + 4 * (k - 13));  // 0..8, 10..16, 20..32
}
static_assert(band_width(kBandNumWidths - 1) == kBandHalo, "the widest band fills the border");

template <typename V>
__device__ __forceinline__ decltype(V::x) win_el(const V* win, int d) {
  return (d & 1) ? win[d >> 1].y : win[d >> 1].x;
}

// Where a banded row's float64 slices go (CPC_FP64_TC): its slice row, and the
// largest |U| of its column, from which the row exponent is bounded before
// any output exists: |W[i]| <= sum_m |p_q[|m|]| max|U|, so each output pair is
// sliced as it is computed (no row reduction, no second pass)
struct BandSlice64 {
  __nv_bfloat16* ob;  // the row in slice 0, chunk 0
  long long stride;   // elements between slices
  int R_f;
  int* expo;          // the row's exponent
  double umax;
};

// outputs i, i+1 for every even i = 2 threadIdx.x + 2 kBandThreads j < n;
// float32 SLICE: also kept in ws, and this thread's largest |W| returned;
// float64 SLICE: the digits written as computed
template <typename T, int H, bool SLICE>
__device__ __forceinline__ T band_rows(const T* __restrict__ us, int n, const void* __restrict__ taps_q,
                                       T* __restrict__ w, T* __restrict__ ws, const BandSlice64& b64) {
  using V = typename cvec<T>::type;
  constexpr int H2 = (H + 1) & ~1;  // the window starts at an even cell
  constexpr int HL = (H + 1) / 2;   // float32: taps with their lo part
  T ph[H + 1];
  float pl[HL + 1];
  if constexpr (sizeof(T) == 4) {
    const float2* tp = static_cast<const float2*>(taps_q);
#pragma unroll
    for (int m = 0; m <= H; ++m) {
      const float2 v = __ldg(tp + m);
      ph[m] = v.x;
      if (m <= HL) pl[m] = v.y;
    }
  } else {
    const double* tp = static_cast<const double*>(taps_q);
#pragma unroll
    for (int m = 0; m <= H; ++m) ph[m] = __ldg(tp + m);
  }
  int e64 = 0;
  if constexpr (SLICE && sizeof(T) == 8) if (b64.ob) {  // (NULL: a lag-covered term, no slices)
    // the float64 sum of 2H + 1 products stays below the bound times
    // (1 + (2H + 2) 2^-53); 2^e above the bound times (1 + 2^-40)
    double S = fabs(ph[0]);
#pragma unroll
    for (int m = 1; m <= H; ++m) S += 2.0 * fabs(ph[m]);
    e64 = row_exponent64(biased_exponent64(S * b64.umax * (1.0 + 0x1p-40)));
    if (threadIdx.x == 0) *b64.expo = e64;
  }
  T mx = T(0);
  for (int i = 2 * threadIdx.x; i < n; i += 2 * kBandThreads) {
    // cells i - H2 .. i + H2 + 1
    const V* u2 = reinterpret_cast<const V*>(us + kBandHalo + i - H2);
    V win[H2 + 1];
#pragma unroll
    for (int d = 0; d <= H2; ++d) win[d] = u2[d];
    T a0 = T(0), a1 = T(0);
    float l0 = 0.0f, l1 = 0.0f;
    // smallest taps first
#pragma unroll
    for (int m = H; m >= 1; --m) {
      const T s0 = win_el(win, H2 - m) + win_el(win, H2 + m);
      const T s1 = win_el(win, H2 + 1 - m) + win_el(win, H2 + 1 + m);
      if constexpr (sizeof(T) == 4) {
        a0 = fmaf(ph[m], s0, a0);
        a1 = fmaf(ph[m], s1, a1);
        if (m <= HL) {
          l0 = fmaf(pl[m], s0, l0);
          l1 = fmaf(pl[m], s1, l1);
        }
      } else {
        a0 = fma(ph[m], s0, a0);
        a1 = fma(ph[m], s1, a1);
      }
    }
    if constexpr (sizeof(T) == 4) {
      a0 = fmaf(ph[0], win_el(win, H2), a0) + fmaf(pl[0], win_el(win, H2), l0);
      a1 = fmaf(ph[0], win_el(win, H2 + 1), a1) + fmaf(pl[0], win_el(win, H2 + 1), l1);
    } else {
      a0 = fma(ph[0], win_el(win, H2), a0);
      a1 = fma(ph[0], win_el(win, H2 + 1), a1);
    }
    __stcs(reinterpret_cast<V*>(w + i), cmk<V>(a0, a1));
    if constexpr (SLICE) {
      if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<V*>(ws + i) = cmk<V>(a0, a1);
        mx = fmaxf(mx, fmaxf(fabsf(a0), fabsf(a1)));
      } else if (b64.ob) {
        constexpr int C = kSlice64Cells;
        slice64_pair(a0, a1, e64, b64.ob + (long long)(i / C) * b64.R_f * C + (i % C), b64.stride);
      }
    }
  }
  return mx;
}

template <typename T, bool SLICE, int K = 0>
__device__ __forceinline__ T band_dispatch(int h, const T* us, int n, const void* tq, T* w, T* ws,
                                           const BandSlice64& b64) {
  if constexpr (K == kBandNumWidths - 1) {
    return band_rows<T, band_width(K), SLICE>(us, n, tq, w, ws, b64);  // the widest (and any unknown) width
  } else {
    if (h == band_width(K)) return band_rows<T, band_width(K), SLICE>(us, n, tq, w, ws, b64);
    return band_dispatch<T, SLICE, K + 1>(h, us, n, tq, w, ws, b64);
  }
}

// Double-float arithmetic for the float64-accurate forms CPC_SPLIT and
// CPC_FP64_TC (dfloat.cuh; the float64 pipe of this GPU runs at 1/64 of the
// float32 rate): a product of a double-float tap or coefficient with a
// double-float value, taken as hi + lo (the exact error of the leading
// product by the fused multiply-add plus the cross terms), added to a running
// sum kept as a TwoSum hi part and a float lo part; the sum is rounded to
// float64 once at the end.  About 2^-47 of each product; at most 33 products.
__device__ __forceinline__ void df_acc(float& h, float& l, float2 p, float sh, float sl) {
  const float pr = p.x * sh;
  const float e = fmaf(p.x, sl, fmaf(p.y, sh, fmaf(p.x, sh, -pr)));
  const float t = h + pr, v = t - h;
  l += ((h - (t - v)) + (pr - v)) + e;
  h = t;
}
// a + b of two double-float values (TwoSum of the hi parts, the lo parts added)
__device__ __forceinline__ float2 df_add2(float2 a, float2 b) {
  const float s = a.x + b.x, v = s - a.x;
  return make_float2(s, ((a.x - (s - v)) + (b.x - v)) + (a.y + b.y));
}

// The banded sum in double-float: the column staged as (hi, lo) pairs, taps
// p_q[m] as the float32 class's (hi, lo) pairs, W written in float64 and, for
// CPC_FP64_TC, sliced as computed (BandSlice64) with the row exponent from the
// bound sum_m |p_q[m]| max|U|, here summed in float32 with a 2^-16 margin.
template <int H, bool SLICE>
__device__ __forceinline__ void band_rows_df(const float2* __restrict__ us, int n, const float2* __restrict__ tp,
                                             double* __restrict__ w, const BandSlice64& b64) {
  float2 p[H + 1];
#pragma unroll
  for (int m = 0; m <= H; ++m) p[m] = __ldg(tp + m);
  int e64 = 0;
  if constexpr (SLICE) if (b64.ob) {
    float S = fabsf(p[0].x);
#pragma unroll
    for (int m = 1; m <= H; ++m) S += 2.0f * fabsf(p[m].x);
    e64 = row_exponent64(biased_exponent64(double(S) * b64.umax * (1.0 + 0x1p-16)));
    if (threadIdx.x == 0) *b64.expo = e64;
  }
  for (int i = 2 * threadIdx.x; i < n; i += 2 * kBandThreads) {
    // cells i - H .. i + 1 + H, read from shared memory (a register window of
    // 2 H + 2 pairs would spill)
    const float2* u = us + kBandHalo + i;
    float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
    // smallest taps first
#pragma unroll
    for (int m = H; m >= 1; --m) {
      const float2 s0 = df_add2(u[-m], u[m]);
      const float2 s1 = df_add2(u[1 - m], u[1 + m]);
      df_acc(h0, l0, p[m], s0.x, s0.y);
      df_acc(h1, l1, p[m], s1.x, s1.y);
    }
    const float2 c0 = u[0], c1 = u[1];
    df_acc(h0, l0, p[0], c0.x, c0.y);
    df_acc(h1, l1, p[0], c1.x, c1.y);
    const double a0 = double_of_float_exact(h0) + double_of_float_exact(l0);
    const double a1 = double_of_float_exact(h1) + double_of_float_exact(l1);
    __stcs(reinterpret_cast<double2*>(w + i), make_double2(a0, a1));
    if constexpr (SLICE) {
      if (b64.ob) {
        constexpr int C = kSlice64Cells;
        slice64_pair(a0, a1, e64, b64.ob + (long long)(i / C) * b64.R_f * C + (i % C), b64.stride);
      }
    }
  }
}

template <bool SLICE, int K = 0>
__device__ __forceinline__ void band_dispatch_df(int h, const float2* us, int n, const float2* tq, double* w,
                                                 const BandSlice64& b64) {
  if constexpr (K == kBandNumWidths - 1) {
    band_rows_df<band_width(K), SLICE>(us, n, tq, w, b64);
  } else {
    if (h == band_width(K)) return band_rows_df<band_width(K), SLICE>(us, n, tq, w, b64);
    band_dispatch_df<SLICE, K + 1>(h, us, n, tq, w, b64);
  }
}

// U: [ncols][n] float64 factor columns; items (col, j), j < n_band, term
// qlist[j] with half-width hq[qlist[j]] (a value of band_width); taps:
// [R_N][kBandTaps] (float32 W and DF: float2 (hi, lo), float64 W: double); W
// row col R_N + q.  DF (float64 W only): double-float arithmetic
// (band_rows_df), the column staged as (hi, lo) pairs.
template <typename T, bool SLICE, bool DF = false>
__global__ void __launch_bounds__(kBandThreads, 2)
band_conv_kernel(const double* __restrict__ U, int n, int ncols, int R_N, const int* __restrict__ qlist, int n_band,
                 const int* __restrict__ hq, const void* __restrict__ taps, T* __restrict__ W, SliceOut so,
                 int slice_min_h) {
  using V = typename cvec<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* us = reinterpret_cast<T*>(smem_raw);  // [kBandHalo + n + kBandHalo]
  T* ws = reinterpret_cast<T*>(smem_raw + sizeof(T) * (size_t(n) + 2 * kBandHalo));  // SLICE, float32: [n]
  __shared__ T red[2][kBandThreads / 32];
  __shared__ double ured[kBandThreads / 32];
  double umax = 0.0;  // float64 SLICE: largest |U| of the staged column
  for (int k = threadIdx.x; k < kBandHalo; k += kBandThreads) {
    us[k] = T(0);
    us[kBandHalo + n + k] = T(0);
  }
  const long long n_items = (long long)ncols * n_band;
  const long long k0 = n_items * blockIdx.x / gridDim.x;
  const long long k1 = n_items * (blockIdx.x + 1) / gridDim.x;
  long long staged = -1;
  int parity = 0;
  long long col = k0 / n_band;
  int jq = int(k0 - col * n_band);
  for (long long k = k0; k < k1; ++k, (++jq == n_band ? (jq = 0, ++col) : 0)) {
    const int q = __ldg(qlist + jq);
    if (col != staged) {
      __syncthreads();  // every reader of the previous column is done
      const double2* src = reinterpret_cast<const double2*>(U + (size_t)col * n);
      double um = 0.0;
      for (int j = threadIdx.x; j < n / 2; j += kBandThreads) {
        const double2 v = src[j];
        if constexpr (DF) {
          const df d0(v.x), d1(v.y);
          *reinterpret_cast<float4*>(reinterpret_cast<float2*>(us) + kBandHalo + 2 * j) =
              make_float4(d0.hi, d0.lo, d1.hi, d1.lo);
        } else {
          *reinterpret_cast<V*>(us + kBandHalo + 2 * j) = cmk<V>(T(v.x), T(v.y));
        }
        if constexpr (SLICE && sizeof(T) == 8) um = fmax(um, fmax(fabs(v.x), fabs(v.y)));
      }
      if constexpr (SLICE && sizeof(T) == 8) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
        if ((threadIdx.x & 31) == 0) ured[threadIdx.x >> 5] = um;
      }
      staged = col;
      __syncthreads();
      if constexpr (SLICE && sizeof(T) == 8) {
        umax = ured[0];
#pragma unroll
        for (int w = 1; w < kBandThreads / 32; ++w) umax = fmax(umax, ured[w]);
      }
    }
    const long long item = col * R_N + q;
    const void* tq = (sizeof(T) == 4) ? static_cast<const void*>(static_cast<const float2*>(taps) + (size_t)q * kBandTaps)
                                      : static_cast<const void*>(static_cast<const double*>(taps) + (size_t)q * kBandTaps);
    const int h = __ldg(hq + q);
    BandSlice64 b64{nullptr, 0, 0, nullptr, umax};
    if constexpr (SLICE && sizeof(T) == 8) if (h >= slice_min_h) {
      constexpr int C = kSlice64Cells;
      const int l = int(col / so.R_f), srow = int(col - (long long)l * so.R_f);
      b64 = BandSlice64{so.out + ((long long)(l * R_N + q) * (n / C) * so.R_f + srow) * C, so.slice_stride, so.R_f,
                        so.expo + item, umax};
    }
    T mx = T(0);
    if constexpr (DF) {
      static_assert(sizeof(T) == 8, "double-float banded sums write float64 W");
      band_dispatch_df<SLICE>(h, reinterpret_cast<const float2*>(us), n,
                              static_cast<const float2*>(taps) + (size_t)q * kBandTaps, W + (size_t)item * n, b64);
    } else {
      mx = band_dispatch<T, SLICE>(h, us, n, tq, W + (size_t)item * n, ws, b64);
    }
    // float32: the terms with H < slice_min_h get no slices (their Gram
    // matrices come from the lag Gram matrices); h is the same for the CTA
    if constexpr (SLICE && sizeof(T) == 4) if (h >= slice_min_h) {
      // row maximum over the CTA (red is double-buffered: one barrier per item)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((threadIdx.x & 31) == 0) red[parity][threadIdx.x >> 5] = mx;
      __syncthreads();
      T m = red[parity][0];
#pragma unroll
      for (int w = 1; w < kBandThreads / 32; ++w) m = fmax(m, red[parity][w]);
      parity ^= 1;
      const int l = int(col / so.R_f), srow = int(col - (long long)l * so.R_f);
      const int e = balanced_exponent(m);
      if (threadIdx.x == 0) so.expo[item] = e;
      __nv_bfloat16* ob = so.out + ((long long)(l * R_N + q) * (n / 64) * so.R_f + srow) * 64;
      float sc1, sc2;
      slice_scales(e, sc1, sc2);
      // this thread's own outputs (no barrier needed for ws)
      for (int i = 2 * threadIdx.x; i < n; i += 2 * kBandThreads) {
        const float2 v = *reinterpret_cast<const float2*>(ws + i);
        slice_pair(v.x, v.y, sc1, sc2, ob + (long long)(i >> 6) * so.R_f * 64 + (i & 63), so.slice_stride);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Separable Chebyshev form of the smooth kernel terms (Sec. 2.5, Eq. conv).
// A term with a small exponent t_q varies slowly across the whole box: on
// [-b, b]^2 the kernel g_q(x, y) = f_q(x - y) (f_q(m h) = p_q[m], the cell
// integral of the term's Gaussian) is, to a set fraction of f_q(0) (2^-34 for
// float32 W, 2^-46 for float64 W, checked on the grid by the host; float64
// evaluation noise of the check itself is near 2^-50), the polynomial
// sum_{k,l<K} C_kl T_k(x/b) T_l(y/b).  Then
//   W[i] = sum_j g_q(x_i, x_j) U[j] = sum_k d_k T_k(x_i/b),
//   d_k  = sum_l C_kl m_l,  m_l = sum_j T_l(x_j/b) U[j],
// so each convolution costs K multiply-adds per output once the K moments of
// its column are known (they are shared by all smooth terms).
//   cheb_moments_kernel: m_l of every column;
//   cheb_coef_kernel: d = C_q m per (column, term) in float64, stored in the
//     W type (and kept in float64 with the summed moments, for the Gram
//     matrices of cheb_gram_kernel), with a record per item: its W row and
//     its rank;
//   cheb_eval_kernel: W[i] = sum_k d_k T_k(x_i/b) with the thread's table
//     entries in registers, CTAs over 512-cell blocks x item ranges.
constexpr int kCheb = 16;  // largest rank (ranks are 4, 8, 12 or 16)
constexpr int kChebThreads = 256;
// per (column, smooth term): where its W row starts and its rank, computed
// once by cheb_coef_kernel
struct __align__(16) ChebItem {
  long long w_off;  // element offset of the W row
  int K;
  int pad;
};

// Moments as a small GEMM, Mom = T (kCheb x n) U^T (n x ncols): a CTA takes
// 64 columns and a range of kChebCells cells (blockIdx.y), stages the table
// rows and the columns (rounded to T) of CH cells at a time in shared memory,
// and each thread accumulates 4 columns of one k (float32 class: products
// with the (hi, lo) table summed without loss by TwoSum within a stage and
// flushed into float64 once per stage: the moments are shared by every smooth
// term of a column, so their rounding would not average out, and float64
// arithmetic is scarce on this GPU).  Partial moments of every cell range go
// to Part[range][col][k] and are summed by cheb_coef_kernel.
constexpr int kChebCols = 64;
constexpr int kChebCells = 512;
__host__ __device__ constexpr int cheb_ranges(int n) { return n > kChebCells ? n / kChebCells : 1; }

template <typename T>
__global__ void __launch_bounds__(kChebThreads)
cheb_moments_kernel(const double* __restrict__ U, int n, int ncols, const void* __restrict__ tcheb,
                    double* __restrict__ Part) {
  using V = typename cvec<T>::type;
  constexpr int CH = sizeof(T) == 4 ? 64 : 32;        // cells per stage
  __shared__ __align__(16) V ts[kCheb][CH];           // float32 class: (hi, lo); float64: (T, unused)
  __shared__ __align__(16) T us[CH][kChebCols + 4];    // [cell][column], padded
  const int t = threadIdx.x;
  const int k = t / 16, c4 = 4 * (t % 16);              // this thread: moment k of columns c4..c4+3
  const int col0 = blockIdx.x * kChebCols;
  const int cells = n / cheb_ranges(n);
  const int j0 = blockIdx.y * cells;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int jb = j0; jb < j0 + cells; jb += CH) {
    const int w = min(CH, j0 + cells - jb);
    __syncthreads();  // the previous stage is consumed
    for (int x = t; x < kCheb * CH; x += kChebThreads) {
      const int kk = x / CH, jj = x % CH;
      if (jj < w) {
        if constexpr (sizeof(T) == 4) ts[kk][jj] = __ldg(static_cast<const float2*>(tcheb) + (size_t)kk * n + jb + jj);
        else ts[kk][jj] = make_double2(__ldg(static_cast<const double*>(tcheb) + (size_t)kk * n + jb + jj), 0.0);
      }
    }
    for (int x = t; x < kChebCols * CH; x += kChebThreads) {
      const int cc = x / CH, jj = x % CH;
      const int c = col0 + cc;
      us[jj][cc] = (c < ncols && jj < w) ? T(__ldg(U + (size_t)c * n + jb + jj)) : T(0);
    }
    __syncthreads();
    if constexpr (sizeof(T) == 4) {
      // per column an unevaluated sum s + e of the stage's products
      // (TwoSum, Knuth), flushed into float64 at the end of the stage
      float sm[4] = {0.f, 0.f, 0.f, 0.f}, er[4] = {0.f, 0.f, 0.f, 0.f};
      for (int jj = 0; jj < w; ++jj) {
        const V tk = ts[k][jj];
        const float4 v = *reinterpret_cast<const float4*>(&us[jj][c4]);
        const float u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float p = fmaf(tk.x, u[m], tk.y * u[m]);
          const float t2 = sm[m] + p;
          const float bp = t2 - sm[m];
          er[m] += (sm[m] - (t2 - bp)) + (p - bp);
          sm[m] = t2;
        }
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] += double(sm[m]) + double(er[m]);
    } else {
      for (int jj = 0; jj < w; ++jj) {
        const V tk = ts[k][jj];
#pragma unroll
        for (int m = 0; m < 4; ++m) acc[m] = fma(tk.x, us[jj][c4 + m], acc[m]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int c = col0 + c4 + m;
    if (c < ncols) Part[((size_t)blockIdx.y * ncols + c) * kCheb + k] = acc[m];
  }
}

// one CTA per column: the moments summed over the cell ranges once (kept in
// Mom[col][kCheb] as double-float pairs), then one thread per smooth term j:
// d_k for k < K (zero up to kCheb) into D[col n_smooth + j][kCheb] (and Ddf as
// double-float pairs) and the item's record
constexpr int kChebCoefThreads = 64;
template <typename T>
__global__ void __launch_bounds__(kChebCoefThreads)
cheb_coef_kernel(int n, int ncols, int R_N, const int* __restrict__ qlist, int n_smooth, const int* __restrict__ kq,
                 const double* __restrict__ cheb, const double* __restrict__ Part, T* __restrict__ D,
                 ChebItem* __restrict__ items, float2* __restrict__ Mom, float2* __restrict__ Ddf) {
  const int col = blockIdx.x;
  __shared__ double m[kCheb];
  if (threadIdx.x < kCheb) {
    double acc = 0.0;
    for (int r = 0; r < cheb_ranges(n); ++r) acc += Part[((size_t)r * ncols + col) * kCheb + threadIdx.x];
    m[threadIdx.x] = acc;
    const df a(acc);  // for the Gram matrices (cheb_gram_kernel), as double-float pairs
    Mom[(size_t)col * kCheb + threadIdx.x] = make_float2(a.hi, a.lo);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n_smooth; j += kChebCoefThreads) {
    const int q = __ldg(qlist + j);
    const int K = __ldg(kq + q);
    const double* C = cheb + (size_t)q * kCheb * kCheb;
    const long long k = (long long)col * n_smooth + j;
    for (int r = 0; r < kCheb; ++r) {
      double d = 0.0;
      if (r < K)
        for (int l = 0; l < K; ++l) d = fma(__ldg(C + r * kCheb + l), m[l], d);
      D[k * kCheb + r] = T(d);
      const df dd(d);
      Ddf[k * kCheb + r] = make_float2(dd.hi, dd.lo);
    }
    ChebItem it;
    it.w_off = ((long long)col * R_N + q) * n;
    it.K = K;
    it.pad = 0;
    items[k] = it;
  }
}

template <typename T, int K>
__device__ __forceinline__ void cheb_pair(const typename cvec<T>::type* dk, const float4* t32, const double2* t64,
                                          T& w0, T& w1) {
  // dk: the item's coefficients as pairs (d_2r, d_2r+1); smallest terms first
  if constexpr (sizeof(T) == 4) {
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int r = K / 2 - 1; r >= 0; --r) {
      const float2 d = dk[r];
      // (hi, lo) of T_k at cells i (x, y) and i+1 (z, w)
      a0 = fmaf(t32[2 * r + 1].x, d.y, fmaf(t32[2 * r + 1].y, d.y, a0));
      a1 = fmaf(t32[2 * r + 1].z, d.y, fmaf(t32[2 * r + 1].w, d.y, a1));
      a0 = fmaf(t32[2 * r].x, d.x, fmaf(t32[2 * r].y, d.x, a0));
      a1 = fmaf(t32[2 * r].z, d.x, fmaf(t32[2 * r].w, d.x, a1));
    }
    w0 = a0;
    w1 = a1;
  } else {
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int r = K / 2 - 1; r >= 0; --r) {
      const double2 d = dk[r];
      a0 = fma(t64[2 * r + 1].x, d.y, a0);
      a1 = fma(t64[2 * r + 1].y, d.y, a1);
      a0 = fma(t64[2 * r].x, d.x, a0);
      a1 = fma(t64[2 * r].y, d.x, a1);
    }
    w0 = a0;
    w1 = a1;
  }
}

// the double-float evaluation (float64 W of CPC_SPLIT and CPC_FP64_TC): the
// coefficients as (hi, lo) pairs (dk2[r]: d_2r and d_2r+1), the table as the
// float32 class's (hi, lo) pairs, sums as df_acc, W rounded to float64 once
template <int K>
__device__ __forceinline__ void cheb_pair_df(const float4* dk2, const float4* t32, double& w0, double& w1) {
  float h0 = 0.0f, l0 = 0.0f, h1 = 0.0f, l1 = 0.0f;
#pragma unroll
  for (int r = K / 2 - 1; r >= 0; --r) {
    const float4 d = dk2[r];
    const float2 dh = make_float2(d.z, d.w), dl = make_float2(d.x, d.y);
    df_acc(h0, l0, dh, t32[2 * r + 1].x, t32[2 * r + 1].y);
    df_acc(h1, l1, dh, t32[2 * r + 1].z, t32[2 * r + 1].w);
    df_acc(h0, l0, dl, t32[2 * r].x, t32[2 * r].y);
    df_acc(h1, l1, dl, t32[2 * r].z, t32[2 * r].w);
  }
  w0 = double_of_float_exact(h0) + double_of_float_exact(l0);
  w1 = double_of_float_exact(h1) + double_of_float_exact(l1);
}

// grid: x = 512-cell blocks of the rows, y = ranges of items (col, j); the
// records (d row and header) of kChebBatch items at a time are staged in
// shared memory with coalesced loads, then every thread evaluates its two
// cells for each of them.  DF (float64 W only): D holds the coefficients as
// double-float pairs and tcheb the float32 class's (hi, lo) table.
constexpr int kChebBatch = 32;
template <typename T, bool DF = false>
__global__ void __launch_bounds__(kChebThreads, 2)
cheb_eval_kernel(int n, int ncols, int n_smooth, const void* __restrict__ tcheb, const void* __restrict__ D,
                 const ChebItem* __restrict__ items, T* __restrict__ W) {
  using V = typename cvec<T>::type;
  static_assert(!DF || sizeof(T) == 8, "double-float evaluation writes float64 W");
  __shared__ __align__(16) T sd[kChebBatch][kCheb];  // (DF: kCheb (hi, lo) pairs per row, the same bytes)
  __shared__ ChebItem sh[kChebBatch];
  const int i = blockIdx.x * 2 * kChebThreads + 2 * threadIdx.x;  // cells i, i+1
  const bool on = i < n;
  // this thread's table entries: T_k at cells i and i+1
  float4 t32[sizeof(T) == 4 || DF ? kCheb : 1];
  double2 t64[sizeof(T) == 8 && !DF ? kCheb : 1];
  if constexpr (sizeof(T) == 4 || DF) {
    const float2* tc = static_cast<const float2*>(tcheb);
#pragma unroll
    for (int k = 0; k < kCheb; ++k)
      t32[k] = on ? __ldg(reinterpret_cast<const float4*>(tc + (size_t)k * n + i)) : make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    const double* tc = static_cast<const double*>(tcheb);
#pragma unroll
    for (int k = 0; k < kCheb; ++k)
      t64[k] = on ? __ldg(reinterpret_cast<const double2*>(tc + (size_t)k * n + i)) : make_double2(0.0, 0.0);
  }
  const long long n_items = (long long)ncols * n_smooth;
  const long long k0 = n_items * blockIdx.y / gridDim.y, k1 = n_items * (blockIdx.y + 1) / gridDim.y;
  for (long long kb = k0; kb < k1; kb += kChebBatch) {
    const int nb = int(min((long long)kChebBatch, k1 - kb));
    __syncthreads();  // the previous batch is consumed
    {
      // d rows and records as 16-byte pieces
      constexpr int PIECES = kCheb * sizeof(T) / 16;
      constexpr int RP = sizeof(ChebItem) / 16;
      const uint4* src = reinterpret_cast<const uint4*>(static_cast<const T*>(D) + kb * kCheb);
      uint4* dst = reinterpret_cast<uint4*>(&sd[0][0]);
      for (int x = threadIdx.x; x < nb * PIECES; x += kChebThreads) dst[x] = __ldg(src + x);
      const uint4* isrc = reinterpret_cast<const uint4*>(items + kb);
      uint4* idst = reinterpret_cast<uint4*>(sh);
      for (int x = threadIdx.x; x < nb * RP; x += kChebThreads) idst[x] = __ldg(isrc + x);
    }
    __syncthreads();
    if (!on) continue;
    for (int b = 0; b < nb; ++b) {
      const ChebItem& h = sh[b];
      T w0, w1;
      if constexpr (DF) {
        const float4* dk2 = reinterpret_cast<const float4*>(sd[b]);
        if (h.K <= 4) cheb_pair_df<4>(dk2, t32, w0, w1);
        else if (h.K <= 8) cheb_pair_df<8>(dk2, t32, w0, w1);
        else if (h.K <= 12) cheb_pair_df<12>(dk2, t32, w0, w1);
        else cheb_pair_df<16>(dk2, t32, w0, w1);
      } else {
        const V* dk = reinterpret_cast<const V*>(sd[b]);
        if (h.K <= 4) cheb_pair<T, 4>(dk, t32, t64, w0, w1);
        else if (h.K <= 8) cheb_pair<T, 8>(dk, t32, t64, w0, w1);
        else if (h.K <= 12) cheb_pair<T, 12>(dk, t32, t64, w0, w1);
        else cheb_pair<T, 16>(dk, t32, t64, w0, w1);
      }
      __stcs(reinterpret_cast<V*>(W + h.w_off + i), cmk<V>(w0, w1));
    }
  }
}

// ---------------------------------------------------------------------------
// Gram matrices of the smooth terms (Sec. 3.2, Eq. Factor_Mk_Conv) from their
// separable form: the Chebyshev path writes W_{l,q}[s][i] = sum_k d_{s,k}
// T_k(x_i/b) with d_s = C_q m_s, so
//   G_{l,q}[r][s] = sum_i U_l[r][i] W_{l,q}[s][i] = sum_k m_{r,k} d_{s,k},
// a K-term sum (K <= 16) per entry in place of the n-term cell sum, with the
// moments m_r = sum_i T(x_i/b) U_l[r][i] the convolution formed (of the
// columns as it read them) and the float64 coefficients d.  The sums run in
// double-float arithmetic (relative error near 2^-44 of sum_k |m_k d_k|,
// against 2^-24 for the float32 form's cell contraction; each product is
// taken as hi + lo, the exact error of the leading product by the fused
// multiply-add plus the cross terms, the running sum as a TwoSum hi part and
// a float lo part, added once at the end).  A CTA takes one
// smooth term and one 32 x 32 tile pair (row tile <= column tile) of the
// symmetric G, four entries per thread; with G it writes both triangles, with
// c it sums (1 or 2) c_r c_s prod_l G_l[r][s] over r <= s into one partial
// (the cell contraction's convention).
constexpr int kGramTile = 32;
constexpr int kGramThreads = 256;
__host__ __device__ constexpr int gram_tiles(int R_f) { return (R_f + kGramTile - 1) / kGramTile; }

__global__ void __launch_bounds__(kGramThreads)
cheb_gram_kernel(int R_f, int R_N, const int* __restrict__ smooth_q, int n_smooth, const int* __restrict__ kq,
                 const float2* __restrict__ Mom, const float2* __restrict__ Ddf, const double* __restrict__ c,
                 double* __restrict__ G, double* __restrict__ partial) {
  constexpr int TP = kGramTile + 2;  // padded rows (16-byte aligned for the paired reads)
  __shared__ __align__(16) float2 mr[3][kCheb][TP];  // double-float (hi, lo)
  __shared__ __align__(16) float2 ds[3][kCheb][TP];
  __shared__ double red[kGramThreads / 32];
  const int j = blockIdx.y;
  const int q = __ldg(smooth_q + j);
  const int K = __ldg(kq + q);
  const int nt = gram_tiles(R_f);
  int pi = blockIdx.x, rt = 0;
  while (pi >= nt - rt) {  // pair index -> (row tile, column tile >= row tile)
    pi -= nt - rt;
    ++rt;
  }
  const int st = rt + pi;
  const int r0 = rt * kGramTile, s0 = st * kGramTile;
  // the tile's moments and coefficients, rows of kCheb float64 read whole
  for (int x = threadIdx.x; x < 3 * kGramTile * kCheb; x += kGramThreads) {
    const int k = x % kCheb, i = (x / kCheb) % kGramTile, l = x / (kCheb * kGramTile);
    const int r = r0 + i, sc = s0 + i;
    const float2 z = make_float2(0.0f, 0.0f);
    mr[l][k][i] = (r < R_f && k < K) ? __ldg(Mom + (size_t)(l * R_f + r) * kCheb + k) : z;
    ds[l][k][i] = (sc < R_f && k < K) ? __ldg(Ddf + ((size_t)(l * R_f + sc) * n_smooth + j) * kCheb + k) : z;
  }
  __syncthreads();
  const int tr = threadIdx.x / 8, ts = 4 * (threadIdx.x % 8);
  const int r = r0 + tr;
  float Gh[3][4], Gl[3][4];  // each entry as the unevaluated sum Gh + Gl
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < K; ++k) {
      const float2 m = mr[l][k][tr];
      const float4 d01 = *reinterpret_cast<const float4*>(&ds[l][k][ts]);
      const float4 d23 = *reinterpret_cast<const float4*>(&ds[l][k][ts + 2]);
      const float dh[4] = {d01.x, d01.z, d23.x, d23.z}, dl[4] = {d01.y, d01.w, d23.y, d23.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float p = m.x * dh[i];
        const float e = fmaf(m.x, dl[i], fmaf(m.y, dh[i], fmaf(m.x, dh[i], -p)));  // the rest of the product
        const float sh = hi[i] + p, v = sh - hi[i];
        lo[i] += ((hi[i] - (sh - v)) + (p - v)) + e;  // TwoSum error of hi + p
        hi[i] = sh;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      Gh[l][i] = hi[i];
      Gl[l][i] = lo[i];
    }
  }
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int sc = s0 + ts + i;
    if (r >= R_f || sc >= R_f || (rt == st && tr > ts + i)) continue;
    if (G) {
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const double gv = double(Gh[l][i]) + double(Gl[l][i]);
        double* Gq = G + ((size_t)l * R_N + q) * R_f * R_f;
        Gq[(size_t)r * R_f + sc] = gv;
        Gq[(size_t)sc * R_f + r] = gv;
      }
    }
    // E_H: the product over axes in float32, the weighted sum in float64 (as the
    // cell contraction forms it)
    if (c) {
      const float pr = (Gh[0][i] + Gl[0][i]) * (Gh[1][i] + Gl[1][i]) * (Gh[2][i] + Gl[2][i]);
      const double cs = __ldg(c + sc);
      sum = fma(r == sc ? cs : 2.0 * cs, double(pr), sum);
    }
  }
  if (!c) return;
  if (r < R_f) sum *= __ldg(c + r);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kGramThreads / 32; ++w) t += red[w];
    partial[(size_t)j * gridDim.x + blockIdx.x] = t;
  }
}

// Rows-mode operands of the smooth terms (the Coulomb matrix): the same
// identity as cheb_gram_kernel, G[r][(m, q)] = sum_k m_{r,k} d_{m,q,k}, taken
// by the tensor-core rows contraction with the kCheb moments and coefficients
// as the "cells" of zero-padded rows.
//   moment_rows_kernel: out[col][k] = sum over cell ranges of Part (k < kCheb), 0 beyond;
//   coef_rows_kernel: out[row][k] = D[row][k] (k < kCheb), 0 beyond.
__global__ void moment_rows_kernel(const double* __restrict__ Part, int ranges, long long ncols, double* __restrict__ out,
                                   int width) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= ncols * width) return;
  const long long col = x / width;
  const int k = int(x - col * width);
  double acc = 0.0;
  if (k < kCheb)
    for (int r = 0; r < ranges; ++r) acc += Part[((size_t)r * ncols + col) * kCheb + k];
  out[x] = acc;
}
__global__ void coef_rows_kernel(const float* __restrict__ D, long long rows, float* __restrict__ out, int width) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= rows * width) return;
  const long long row = x / width;
  const int k = int(x - row * width);
  out[x] = k < kCheb ? D[row * kCheb + k] : 0.0f;
}

// ---------------------------------------------------------------------------
// Gram matrices of the narrow (banded) terms from lag Gram matrices (Sec. 3.2,
// Eq. Factor_Mk_Conv with the banded sum of Eq. conv): with
//   V_m[i] = U[i - m] + U[i + m] (m > 0, zero outside the grid), V_0 = U,
// a banded term's W is sum_{m <= H} p_q[m] V_m, so
//   G_q = U^T W_q = sum_{m <= H} p_q[m] S_m,  S_m = U^T V_m,
// and the L lag Gram matrices S_0..S_{L-1} (contracted over the cells on the
// tensor cores, as extra rows of the float32 energy path) give every banded
// term with H < L.  lag_slice32_kernel writes V_m (the column rounded to
// float32 once, as the banded kernel stages it, then float32 sums: no
// float64 arithmetic, which runs at 1/64 of the float32 rate here) as the
// contraction's balanced three-digit slices into the slice slot of the m-th
// covered term: one CTA per (axis, column) stages the column once in shared
// memory (zero border of kMaxLags cells), takes the L row maxima in one pass
// and writes the L rows' digits in a second.
constexpr int kLagThreads = 256;
__global__ void __launch_bounds__(kLagThreads)
lag_slice32_kernel(const double* __restrict__ U, int n, int R_f, int R_N, int L, const int* __restrict__ slots,
                   SliceOut so) {
  extern __shared__ __align__(16) float ul[];  // [kMaxLags + n + kMaxLags]
  __shared__ float red[kMaxLags][kLagThreads / 32];
  for (int k = threadIdx.x; k < kMaxLags; k += kLagThreads) {
    ul[k] = 0.0f;
    ul[kMaxLags + n + k] = 0.0f;
  }
  float* u = ul + kMaxLags;
  for (long long col = blockIdx.x; col < 3LL * R_f; col += gridDim.x) {
    __syncthreads();  // the previous column is consumed
    const double2* src = reinterpret_cast<const double2*>(U + col * n);
    for (int j = threadIdx.x; j < n / 2; j += kLagThreads) {
      const double2 v = src[j];
      *reinterpret_cast<float2*>(u + 2 * j) = make_float2(float(v.x), float(v.y));
    }
    __syncthreads();
    float mx[kMaxLags];
#pragma unroll
    for (int m = 0; m < kMaxLags; ++m) mx[m] = 0.0f;
    for (int i = threadIdx.x; i < n; i += kLagThreads) {
      mx[0] = fmaxf(mx[0], fabsf(u[i]));
#pragma unroll
      for (int m = 1; m < kMaxLags; ++m)
        if (m < L) mx[m] = fmaxf(mx[m], fabsf(u[i - m] + u[i + m]));
    }
#pragma unroll
    for (int m = 0; m < kMaxLags; ++m) {
      if (m < L) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx[m] = fmaxf(mx[m], __shfl_xor_sync(0xffffffffu, mx[m], o));
        if ((threadIdx.x & 31) == 0) red[m][threadIdx.x >> 5] = mx[m];
      }
    }
    __syncthreads();
    const int l = int(col / R_f), srow = int(col - (long long)l * R_f);
    for (int m = 0; m < L; ++m) {
      float mm = red[m][0];
#pragma unroll
      for (int w = 1; w < kLagThreads / 32; ++w) mm = fmaxf(mm, red[m][w]);
      const int q = __ldg(slots + m);
      const int e = balanced_exponent(mm);
      if (threadIdx.x == 0) so.expo[col * R_N + q] = e;
      __nv_bfloat16* ob = so.out + ((long long)(l * R_N + q) * (n / 64) * so.R_f + srow) * 64;
      float sc1, sc2;
      slice_scales(e, sc1, sc2);
      for (int i = 2 * threadIdx.x; i < n; i += 2 * kLagThreads) {
        const float v0 = m ? u[i - m] + u[i + m] : u[i];
        const float v1 = m ? u[i + 1 - m] + u[i + 1 + m] : u[i + 1];
        slice_pair(v0, v1, sc1, sc2, ob + (long long)(i >> 6) * so.R_f * 64 + (i & 63), so.slice_stride);
      }
    }
  }
}

// The float64 form's lag rows (FP64_TC): V_m in float64 (one addition per
// cell), sliced into the five weighted digits of the float64 form with the
// row's largest exponent field, into the slot of the m-th covered term; a CTA
// per (axis, column) stages the column in shared memory as lag_slice32_kernel.
__global__ void __launch_bounds__(kLagThreads)
lag_slice64_kernel(const double* __restrict__ U, int n, int R_f, int R_N, int L, const int* __restrict__ slots,
                   SliceOut so) {
  extern __shared__ __align__(16) double ud[];  // [kMaxLags + n + kMaxLags]
  __shared__ int red[kMaxLags][kLagThreads / 32];
  constexpr int C = kSlice64Cells;
  for (int k = threadIdx.x; k < kMaxLags; k += kLagThreads) {
    ud[k] = 0.0;
    ud[kMaxLags + n + k] = 0.0;
  }
  double* u = ud + kMaxLags;
  for (long long col = blockIdx.x; col < 3LL * R_f; col += gridDim.x) {
    __syncthreads();  // the previous column is consumed
    const double2* src = reinterpret_cast<const double2*>(U + col * n);
    for (int j = threadIdx.x; j < n / 2; j += kLagThreads) *reinterpret_cast<double2*>(u + 2 * j) = src[j];
    __syncthreads();
    int mb[kMaxLags];
#pragma unroll
    for (int m = 0; m < kMaxLags; ++m) mb[m] = 0;
    for (int i = threadIdx.x; i < n; i += kLagThreads) {
      mb[0] = max(mb[0], biased_exponent64(u[i]));
#pragma unroll
      for (int m = 1; m < kMaxLags; ++m)
        if (m < L) mb[m] = max(mb[m], biased_exponent64(u[i - m] + u[i + m]));
    }
#pragma unroll
    for (int m = 0; m < kMaxLags; ++m) {
      if (m < L) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mb[m] = max(mb[m], __shfl_xor_sync(0xffffffffu, mb[m], o));
        if ((threadIdx.x & 31) == 0) red[m][threadIdx.x >> 5] = mb[m];
      }
    }
    __syncthreads();
    const int l = int(col / R_f), srow = int(col - (long long)l * R_f);
    for (int m = 0; m < L; ++m) {
      int mm = red[m][0];
#pragma unroll
      for (int w = 1; w < kLagThreads / 32; ++w) mm = max(mm, red[m][w]);
      const int q = __ldg(slots + m);
      const int e = row_exponent64(mm);
      if (threadIdx.x == 0) so.expo[col * R_N + q] = e;
      __nv_bfloat16* ob = so.out + ((long long)(l * R_N + q) * (n / C) * so.R_f + srow) * C;
      for (int i = 2 * threadIdx.x; i < n; i += 2 * kLagThreads) {
        const double v0 = m ? u[i - m] + u[i + m] : u[i];
        const double v1 = m ? u[i + 1 - m] + u[i + 1 + m] : u[i + 1];
        slice64_pair(v0, v1, e, ob + (long long)(i / C) * so.R_f * C + (i % C), so.slice_stride);
      }
    }
  }
}

// FP64_TC: G_q = sum_{m <= H_q} p_q[m] S_m of the covered terms in float64
// into G (both triangles), for the E_H sum over G that follows
__global__ void __launch_bounds__(kGramThreads)
lag_gram64_kernel(int R_f, int R_N, int L, const int* __restrict__ cov, const int* __restrict__ hq,
                  const double* __restrict__ taps, const double* __restrict__ S, double* __restrict__ G) {
  const int q = __ldg(cov + blockIdx.y);
  const int H = __ldg(hq + q);
  const int nt = gram_tiles(R_f);
  int pi = blockIdx.x, rt = 0;
  while (pi >= nt - rt) {
    pi -= nt - rt;
    ++rt;
  }
  const int st = rt + pi;
  double p[kMaxLags];
#pragma unroll
  for (int m = 0; m < kMaxLags; ++m) p[m] = (m <= H && m < L) ? __ldg(taps + (size_t)q * kBandTaps + m) : 0.0;
  const size_t plane = (size_t)R_f * R_f;
  for (int x = threadIdx.x; x < kGramTile * kGramTile; x += kGramThreads) {
    const int r = rt * kGramTile + x / kGramTile, sc = st * kGramTile + x % kGramTile;
    if (r >= R_f || sc >= R_f || (rt == st && r > sc)) continue;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      double g = 0.0;
#pragma unroll
      for (int m = 0; m < kMaxLags; ++m)
        if (m <= H && m < L) g = fma(p[m], S[((size_t)l * L + m) * plane + (size_t)r * R_f + sc], g);
      double* Gq = G + ((size_t)l * R_N + q) * plane;
      Gq[(size_t)r * R_f + sc] = g;
      Gq[(size_t)sc * R_f + r] = g;
    }
  }
}

// A float64 that holds a float32 value exactly, as float32, by integer work on
// its IEEE-754 fields (sign, exponent rebiased from 1023 to 127, the top 23
// mantissa bits): no float64 instruction, whose rate here is 1/64 of
// float32.  Values below the float32 normal range (2^-126) are taken as zero.
__device__ __forceinline__ float float_of_exact_double(double d) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  const unsigned hi = unsigned(b >> 32);
  const int e = int((hi >> 20) & 0x7FFu);
  if (e <= 896) return 0.0f;
  return __uint_as_float((hi & 0x80000000u) | (unsigned(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) |
                         unsigned((b & 0xFFFFFFFFull) >> 29));
}

// G_q = sum_{m <= H_q} p_q[m] S_m for the covered terms, in float32 as the
// cell contraction forms G (S_m are its float32 values, stored as float64;
// the taps p_q[m] are (hi, lo) pairs as in the banded kernel), the product
// over axes in float32 and the weighted sum in float64, as in the cell
// contraction: one covered
// term and one 32 x 32 tile pair (row tile <= column tile) per CTA; E_H
// partials in the cell contraction's convention (with c) and G (when given)
__global__ void __launch_bounds__(kGramThreads)
lag_gram_kernel(int R_f, int R_N, int L, const int* __restrict__ cov, const int* __restrict__ hq,
                const float2* __restrict__ taps, const double* __restrict__ S, const double* __restrict__ c,
                double* __restrict__ G, double* __restrict__ partial) {
  __shared__ double red[kGramThreads / 32];
  const int j = blockIdx.y;
  const int q = __ldg(cov + j);
  const int H = __ldg(hq + q);
  const int nt = gram_tiles(R_f);
  int pi = blockIdx.x, rt = 0;
  while (pi >= nt - rt) {
    pi -= nt - rt;
    ++rt;
  }
  const int st = rt + pi;
  float2 p[kMaxLags];
#pragma unroll
  for (int m = 0; m < kMaxLags; ++m)
    p[m] = (m <= H && m < L) ? __ldg(taps + (size_t)q * kBandTaps + m) : make_float2(0.0f, 0.0f);
  const size_t plane = (size_t)R_f * R_f;
  double sum = 0.0;
  for (int x = threadIdx.x; x < kGramTile * kGramTile; x += kGramThreads) {
    const int r = rt * kGramTile + x / kGramTile, sc = st * kGramTile + x % kGramTile;
    if (r >= R_f || sc >= R_f || (rt == st && r > sc)) continue;
    float prod = 1.0f;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      float g = 0.0f;
#pragma unroll
      for (int m = 0; m < kMaxLags; ++m)
        if (m <= H && m < L) {
          const float sv = float_of_exact_double(S[((size_t)l * L + m) * plane + (size_t)r * R_f + sc]);
          g = fmaf(p[m].x, sv, fmaf(p[m].y, sv, g));
        }
      if (G) {
        double* Gq = G + ((size_t)l * R_N + q) * plane;
        Gq[(size_t)r * R_f + sc] = g;
        Gq[(size_t)sc * R_f + r] = g;
      }
      prod *= g;
    }
    if (c) sum += (r == sc ? 1.0 : 2.0) * __ldg(c + r) * __ldg(c + sc) * double(prod);
  }
  if (!c) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kGramThreads / 32; ++w) t += red[w];
    partial[(size_t)j * gridDim.x + blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------
// The FFT terms of CPC_SPLIT and CPC_FP64_TC in double-float arithmetic
// (dfloat.cuh): the same transform as conv_kernel<double> (float64 plan,
// per-pass twiddles, half-angle step), with every table and the factor
// spectra as double-float pairs, so the transform runs on the float32 pipes;
// W is written in float64.  Error of the transform about 1e-13 relative
// (13 levels of double-float operations), far below the float64 forms' 1e-10
// bar; CPC_FP64 keeps the float64 transform.
template <int LOGN, bool SLICE>
__global__ void __launch_bounds__(Geometry<LOGN, double>::threads, Geometry<LOGN, double>::min_blocks)
conv_df_kernel(const dfc* __restrict__ Uhat, const df* __restrict__ phat, const dfc* __restrict__ hw,
               const dfc* __restrict__ tw, double* __restrict__ W, int R_N, int ncols, const int* __restrict__ qlist,
               int n_q, SliceOut so) {
  using V = dfc;
  using G = Geometry<LOGN, double>;
  using PL = typename G::PL;
  constexpr int NC = PL::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int slot = threadIdx.x / PL::TPF;
  const int t = threadIdx.x % PL::TPF;
  V* sbuf = reinterpret_cast<V*>(smem_raw) + slot * padded_len(NC);
  const df scale(1.0 / double(2 * NC));  // a power of two: exact
  const long long n_groups = (long long)((ncols + G::slots - 1) / G::slots) * n_q;
  const long long g_begin = n_groups * blockIdx.x / gridDim.x;
  const long long g_end = n_groups * (blockIdx.x + 1) / gridDim.x;
  for (long long g = g_begin; g < g_end; ++g) {
    const long long cb = g / n_q;
    const int qi = int(g - cb * n_q);
    const int q = qlist ? __ldg(qlist + qi) : qi;
    const long long colr = cb * G::slots + slot;
    const bool active = colr < ncols;
    const long long col = active ? colr : ncols - 1;
    const long long item = col * R_N + q;
    const V* Uc = Uhat + (size_t)col * (NC + 1);
    const float2* pq = reinterpret_cast<const float2*>(phat) + (size_t)q * (NC + 1);
    {
      // Z'[f] = (A + B) + i e^{+2 pi i f/2n} (A - B), A = Y[f], B = conj Y[n-f], Y = Uhat * phat
      V v[PL::B1][PL::R1];
      constexpr int stride = NC / PL::R1, nbf = NC / (PL::R1 * PL::B1);
#pragma unroll
      for (int b = 0; b < PL::B1; ++b) {
        const int j = b * nbf + t;
#pragma unroll
        for (int r = 0; r < PL::R1; ++r) {
          const int f = j + r * stride;
          const V uf = ld_tw(Uc + f), ur = ld_tw(Uc + (NC - f));
          const float2 pf2 = __ldg(pq + f), pr2 = __ldg(pq + (NC - f));
          const df pf(pf2.x, pf2.y), pr(pr2.x, pr2.y);
          const V A = cmk<V>(uf.x * pf, uf.y * pf);
          const V B = cmk<V>(ur.x * pr, -(ur.y * pr));
          const V sm = cadd(A, B), d = csub(A, B);
          const V wd = twiddle<+1>(d, hw, nullptr, f);  // e^{+i theta} (A - B)
          v[b][r] = cmk<V>(sm.x - wd.y, sm.y + wd.x);
        }
        dft<PL::R1, +1>(v[b]);
      }
      pass_store<NC, PL::R1, PL::B1>(sbuf, v, t, 1);
    }
    __syncthreads();
    middle_passes<LOGN, G::LOGP, +1>(sbuf, t, tw, nullptr);
    {
      V v[1][PL::P];
      pass_compute<NC, PL::P, 1, +1>(sbuf, v, t, NC / PL::P, tw + pass_table_offset<LOGN, G::LOGP>(PL::NP - 1),
                                     nullptr);
      if constexpr (SLICE) {
        double2 wd[PL::P / 2];
#pragma unroll
        for (int r = 0; r < PL::P / 2; ++r) {
          const V w = cmk<V>(v[0][r].x * scale, v[0][r].y * scale);
          wd[r] = make_double2(w.x.to_double(), w.y.to_double());
        }
        if (active) {
          double* out = W + (size_t)item * NC;
#pragma unroll
          for (int r = 0; r < PL::P / 2; ++r) __stcs(reinterpret_cast<double2*>(out + 2 * (t + r * (NC / PL::P))), wd[r]);
        }
        slice64_epilogue<PL>(wd, reinterpret_cast<double2*>(sbuf), so, item, active, slot, t, R_N);
      } else if (active) {
        double* out = W + (size_t)item * NC;
#pragma unroll
        for (int r = 0; r < PL::P / 2; ++r) {
          const int o = t + r * (NC / PL::P);  // complex output o -> reals 2o, 2o+1
          const V w = cmk<V>(v[0][r].x * scale, v[0][r].y * scale);
          __stcs(reinterpret_cast<double2*>(out + 2 * o), make_double2(w.x.to_double(), w.y.to_double()));
        }
      }
    }
    __syncthreads();
  }
}

// Forward transforms of the factor columns for the double-float forms: the
// float64 plan of spectra_kernel (mode 0) in double-float arithmetic, the
// bins X[f], f = 0..n, written as double-float pairs for conv_df_kernel.
template <int LOGN>
__global__ void __launch_bounds__(Geometry<LOGN>::threads)
spectra_df_kernel(const double* __restrict__ src, int ncols, const dfc* __restrict__ hw, const dfc* __restrict__ tw,
                  dfc* __restrict__ out) {
  using V = dfc;
  using G = Geometry<LOGN>;
  using PL = typename G::PL;
  constexpr int NC = PL::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* sbuf = reinterpret_cast<V*>(smem_raw) + (threadIdx.x / PL::TPF) * padded_len(NC);
  const int slot = threadIdx.x / PL::TPF;
  const int t = threadIdx.x % PL::TPF;
  for (int g = blockIdx.x; g * G::slots < ncols; g += gridDim.x) {
    const int col = g * G::slots + slot;
    const bool active = col < ncols;
    const double* x = src + (size_t)(active ? col : ncols - 1) * NC;
    {
      V v[PL::B1][PL::R1];
      constexpr int stride = NC / PL::R1, nbf = NC / (PL::R1 * PL::B1);
#pragma unroll
      for (int b = 0; b < PL::B1; ++b) {
        const int j = b * nbf + t;
#pragma unroll
        for (int r = 0; r < PL::R1; ++r) {
          const int f = j + r * stride;  // packed pair (x[2f], x[2f+1]), zero beyond n
          V z;
          if (2 * f < NC) {
            const double2 a = *reinterpret_cast<const double2*>(x + 2 * f);
            z.x = df(a.x);
            z.y = df(a.y);
          }
          v[b][r] = z;
        }
        dft<PL::R1, -1>(v[b]);
      }
      pass_store<NC, PL::R1, PL::B1>(sbuf, v, t, 1);
    }
    __syncthreads();
    middle_passes<LOGN, G::LOGP, -1>(sbuf, t, tw, nullptr);
    {
      V v[1][PL::P];
      pass_compute<NC, PL::P, 1, -1>(sbuf, v, t, NC / PL::P, tw + pass_table_offset<LOGN, G::LOGP>(PL::NP - 1),
                                     nullptr);
      __syncthreads();
      pass_store<NC, PL::P, 1>(sbuf, v, t, NC / PL::P);
    }
    __syncthreads();
    if (active) {
      // X[f] = (Z[f] + conj Z[n-f])/2 - (i/2) e^{-i theta} (Z[f] - conj Z[n-f]), f = 0..n
      for (int f = t; f <= NC; f += PL::TPF) {
        const V Zf = sbuf[pad_index(f & (NC - 1))];
        const V Zr = cconj(sbuf[pad_index((NC - f) & (NC - 1))]);
        const V sm = cadd(Zf, Zr), d = csub(Zf, Zr);
        const V wd = cmul(ld_tw(hw + f), d);
        const df h(0.5f, 0.0f);
        V X;
        X.x = h * (sm.x + wd.y);
        X.y = h * (sm.y - wd.x);
        reinterpret_cast<float4*>(out)[(size_t)col * (NC + 1) + f] = make_float4(X.x.hi, X.x.lo, X.y.hi, X.y.lo);
      }
    }
    __syncthreads();
  }
}

__global__ void to_df_copy_kernel(const double* __restrict__ src, float2* __restrict__ dst, long long count) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    const df x(src[k]);
    dst[k] = make_float2(x.hi, x.lo);
  }
}

// ---------------------------------------------------------------------------
template <typename K>
int configure(K kern, size_t smem) {
  CPC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
  return CPC_OK;
}

int sm_count() {
  static int count = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    if (count <= 0) count = 1;
  });
  return count;
}

template <int LOGN>
int launch_spectra(int mode, const double* src, int ncols, double2* o64, float2* o32, double* r64,
                   float* r32, const cpc_kernel* P, cudaStream_t s, float4* o4 = nullptr) {
  using G = Geometry<LOGN>;
  const size_t smem = sizeof(double2) * G::slots * padded_len(1 << LOGN);
  auto kern = spectra_kernel<LOGN>;
  int st = configure(kern, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::threads, smem));
  const int groups = (ncols + G::slots - 1) / G::slots;
  const int grid = std::max(1, std::min(groups, std::max(1, per_sm) * sm_count()));
  const int slot = timing_begin("spectra_kernel", s);
  kern<<<grid, G::threads, smem, s>>>(mode, src, ncols, o64, o32, r64, r32, P->d_hw64, P->d_twp64, o4);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("spectra_kernel");
  return CPC_OK;
}

// how the kernel terms of one precision class are convolved
struct TermSplit {
  const int* fft_q;  // NULL: all terms
  int n_fft;
  const int* band_q;
  int n_band;
  const int* band_h;
  const int* smooth_q;
  int n_smooth;
  const int* smooth_k;
};
TermSplit term_split(const cpc_kernel* P, int cls, const double* U) {
  TermSplit ts{nullptr, P->R_N, nullptr, 0, nullptr, nullptr, 0, nullptr};
  if (U && P->d_terms && P->n_band[cls] + P->n_smooth[cls] > 0) {
    const int R_N = P->R_N;
    const int* b = P->d_terms + (size_t)cls * kTermRows * R_N;
    ts = TermSplit{b + 4 * R_N, R_N - P->n_band[cls] - P->n_smooth[cls], b + 2 * R_N, P->n_band[cls], b,
                   b + 3 * R_N, P->n_smooth[cls], b + R_N};
  }
  return ts;
}

// the Chebyshev path's scratch: partial moments [ranges][ncols][kCheb], item
// records [ncols R_N], coefficients in the W type [ncols R_N][kCheb], then
// for the Gram matrices the summed moments [ncols][kCheb] and the
// coefficients [ncols R_N][kCheb] as double-float pairs
struct SmoothScratch {
  double* Part;
  ChebItem* recs;
  void* D;
  float2* Mom;  // summed moments, double-float pairs
  float2* Ddf;  // coefficients, double-float pairs
};
SmoothScratch smooth_scratch(const cpc_kernel* P, int ncols, const void* scratch, size_t wbytes) {
  unsigned char* sc = static_cast<unsigned char*>(const_cast<void*>(scratch));
  SmoothScratch sm;
  sm.Part = reinterpret_cast<double*>(sc);
  sc += align256(sizeof(double) * size_t(cheb_ranges(P->n)) * ncols * kCheb);
  sm.recs = reinterpret_cast<ChebItem*>(sc);
  sc += align256(sizeof(ChebItem) * size_t(ncols) * P->R_N);
  sm.D = sc;
  sc += align256(sizeof(double) * size_t(ncols) * P->R_N * kCheb);
  sm.Mom = reinterpret_cast<float2*>(sc);
  sc += align256(sizeof(float2) * size_t(ncols) * kCheb);
  sm.Ddf = reinterpret_cast<float2*>(sc);
  return sm;
}

template <typename T, int LOGN, bool SLICE, bool XIN>
int launch_conv(const cpc_kernel* P, int ncols, const void* Uhat, void* W, const SliceOut& so, cudaStream_t s,
                const int* qlist, int n_q) {
  using G = Geometry<LOGN, T>;
  using V = typename cvec<T>::type;
  const size_t smem = sizeof(V) * G::slots * padded_len(1 << LOGN);
  auto kern = conv_kernel<T, LOGN, SLICE, XIN>;
  int st = configure(kern, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::threads, smem));
  const long long groups = (long long)((ncols + G::slots - 1) / G::slots) * n_q;
  const long long grid = std::max(1LL, std::min(groups, (long long)std::max(1, per_sm) * sm_count()));
  const T* phat;
  const V* hw;
  const V* tw;
  const __half2* hwl = nullptr;
  const __half2* twl = nullptr;
  if constexpr (sizeof(T) == 8) {
    phat = P->d_phat64; hw = P->d_hw64; tw = P->d_twp64;
  } else {
    phat = XIN ? reinterpret_cast<const T*>(P->d_pp32) : P->d_phat32;
    hw = P->d_hw32; tw = P->d_twp32;
    hwl = static_cast<const __half2*>(P->d_hw32_lo);
    twl = static_cast<const __half2*>(P->d_twp32_lo);
  }
  const int slot = timing_begin("conv_kernel", s);
  kern<<<int(grid), G::threads, smem, s>>>(static_cast<const V*>(Uhat), phat, hw, tw, hwl, twl,
                                           static_cast<T*>(W), P->R_N, ncols, qlist, n_q, so);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("conv_kernel");
  return CPC_OK;
}

// DF (float64 W): the banded sums in double-float arithmetic
template <typename T, bool SLICE, bool DF = false>
int launch_band(const cpc_kernel* P, int ncols, const double* U, T* W, const SliceOut& so, const TermSplit& ts,
                cudaStream_t s, int slice_min_h = 0) {
  const size_t smem = sizeof(T) * (size_t(P->n) + 2 * kBandHalo) + (SLICE && sizeof(T) == 4 ? sizeof(float) * size_t(P->n) : 0);
  auto kern = band_conv_kernel<T, SLICE, DF>;
  int st = configure(kern, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBandThreads, smem));
  const long long items = (long long)ncols * ts.n_band;
  const long long grid = std::max(1LL, std::min(items, (long long)std::max(1, per_sm) * sm_count()));
  const void* taps = sizeof(T) == 4 || DF ? static_cast<const void*>(P->d_taps32) : static_cast<const void*>(P->d_taps64);
  const int slot = timing_begin("band_conv_kernel", s);
  kern<<<int(grid), kBandThreads, smem, s>>>(U, P->n, ncols, P->R_N, ts.band_q, ts.n_band, ts.band_h, taps, W, so,
                                             slice_min_h);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("band_conv_kernel");
  return CPC_OK;
}

template <int LOGN>
int dispatch_spectra(int logn, int mode, const double* src, int ncols, double2* o64, float2* o32,
                     double* r64, float* r32, const cpc_kernel* P, cudaStream_t s, float4* o4 = nullptr) {
  if constexpr (LOGN > kMaxLogN) {
    return fail(CPC_ERR_UNSUPPORTED, "spectra: n too large");
  } else {
    if (logn == LOGN) return launch_spectra<LOGN>(mode, src, ncols, o64, o32, r64, r32, P, s, o4);
    return dispatch_spectra<LOGN + 1>(logn, mode, src, ncols, o64, o32, r64, r32, P, s, o4);
  }
}

template <int LOGN>
int launch_spectra_df(const double* src, int ncols, dfc* out, const cpc_kernel* P, cudaStream_t s) {
  using G = Geometry<LOGN>;
  const size_t smem = sizeof(dfc) * G::slots * padded_len(1 << LOGN);
  auto kern = spectra_df_kernel<LOGN>;
  int st = configure(kern, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::threads, smem));
  const int groups = (ncols + G::slots - 1) / G::slots;
  const int grid = std::max(1, std::min(groups, std::max(1, per_sm) * sm_count()));
  const int slot = timing_begin("spectra_kernel", s);
  kern<<<grid, G::threads, smem, s>>>(src, ncols, reinterpret_cast<const dfc*>(P->d_hwdf),
                                      reinterpret_cast<const dfc*>(P->d_twdf), out);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("spectra_df_kernel");
  return CPC_OK;
}

template <int LOGN>
int dispatch_spectra_df(int logn, const double* src, int ncols, dfc* out, const cpc_kernel* P, cudaStream_t s) {
  if constexpr (LOGN > kMaxLogN) {
    return fail(CPC_ERR_UNSUPPORTED, "spectra: n too large");
  } else {
    if (logn == LOGN) return launch_spectra_df<LOGN>(src, ncols, out, P, s);
    return dispatch_spectra_df<LOGN + 1>(logn, src, ncols, out, P, s);
  }
}

template <int LOGN>
int launch_spectra32(const double* src, int ncols, float4* o4, const cpc_kernel* P, cudaStream_t s) {
  using G = Geometry<LOGN, float>;
  const size_t smem = sizeof(float2) * G::slots * padded_len(1 << LOGN);
  auto kern = spectra32_kernel<LOGN>;
  int st = configure(kern, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::threads, smem));
  const int groups = (ncols + G::slots - 1) / G::slots;
  const int grid = std::max(1, std::min(groups, std::max(1, per_sm) * sm_count()));
  const int slot = timing_begin("spectra_kernel", s);
  kern<<<grid, G::threads, smem, s>>>(src, ncols, P->d_hw32, static_cast<const __half2*>(P->d_hw32_lo), P->d_opf32,
                                      P->d_twp32, static_cast<const __half2*>(P->d_twp32_lo), o4);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("spectra32_kernel");
  return CPC_OK;
}

template <int LOGN>
int dispatch_spectra32(int logn, const double* src, int ncols, float4* o4, const cpc_kernel* P, cudaStream_t s) {
  if constexpr (LOGN > kMaxLogN) {
    return fail(CPC_ERR_UNSUPPORTED, "spectra: n too large");
  } else {
    if (logn == LOGN) return launch_spectra32<LOGN>(src, ncols, o4, P, s);
    return dispatch_spectra32<LOGN + 1>(logn, src, ncols, o4, P, s);
  }
}

// kernel-term pairs (p^[f], p^[n-f]), f = 0..n-1, float32 [R_N][n]
__global__ void kernel_pairs_kernel(const double* __restrict__ phat64, int R_N, int n, float2* __restrict__ pp) {
  const long long total = (long long)R_N * n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const int q = int(k / n), f = int(k % n);
    const double* ph = phat64 + (size_t)q * (n + 1);
    pp[k] = make_float2(float(ph[f]), float(ph[n - f]));
  }
}

template <typename T, int LOGN, bool SLICE, bool XIN = false>
int dispatch_conv(int logn, const cpc_kernel* P, int ncols, const void* Uhat, void* W, const SliceOut& so,
                  cudaStream_t s, const int* qlist, int n_q) {
  if constexpr (LOGN > kMaxLogN) {
    return fail(CPC_ERR_UNSUPPORTED, "conv: n too large");
  } else {
    if constexpr (SLICE && LOGN < 7) {
      if (logn == LOGN) return fail(CPC_ERR_UNSUPPORTED, "sliced conv: n must be at least 128");
    } else {
      if (logn == LOGN) return launch_conv<T, LOGN, SLICE, XIN>(P, ncols, Uhat, W, so, s, qlist, n_q);
    }
    return dispatch_conv<T, LOGN + 1, SLICE, XIN>(logn, P, ncols, Uhat, W, so, s, qlist, n_q);
  }
}

template <int LOGN, bool SLICE>
int launch_conv_df(const cpc_kernel* P, int ncols, const dfc* Uhat, double* W, const SliceOut& so, cudaStream_t s,
                   const int* qlist, int n_q) {
  using G = Geometry<LOGN, double>;
  const size_t smem = sizeof(dfc) * G::slots * padded_len(1 << LOGN);
  auto kern = conv_df_kernel<LOGN, SLICE>;
  int st = configure(kern, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::threads, smem));
  const long long groups = (long long)((ncols + G::slots - 1) / G::slots) * n_q;
  const long long grid = std::max(1LL, std::min(groups, (long long)std::max(1, per_sm) * sm_count()));
  const int slot = timing_begin("conv_kernel", s);
  kern<<<int(grid), G::threads, smem, s>>>(Uhat, reinterpret_cast<const df*>(P->d_phatdf),
                                           reinterpret_cast<const dfc*>(P->d_hwdf),
                                           reinterpret_cast<const dfc*>(P->d_twdf), W, P->R_N, ncols, qlist, n_q,
                                           so);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("conv_df_kernel");
  return CPC_OK;
}

template <int LOGN, bool SLICE>
int dispatch_conv_df(int logn, const cpc_kernel* P, int ncols, const dfc* Uhat, double* W, const SliceOut& so,
                     cudaStream_t s, const int* qlist, int n_q) {
  if constexpr (LOGN > kMaxLogN) {
    return fail(CPC_ERR_UNSUPPORTED, "conv: n too large");
  } else {
    if constexpr (SLICE && LOGN < 7) {
      if (logn == LOGN) return fail(CPC_ERR_UNSUPPORTED, "sliced conv: n must be at least 128");
    } else {
      if (logn == LOGN) return launch_conv_df<LOGN, SLICE>(P, ncols, Uhat, W, so, s, qlist, n_q);
    }
    return dispatch_conv_df<LOGN + 1, SLICE>(logn, P, ncols, Uhat, W, so, s, qlist, n_q);
  }
}

// DF (float64 W): the evaluation in double-float arithmetic
template <typename T, bool DF = false>
int launch_smooth(const cpc_kernel* P, int ncols, const double* U, T* W, const TermSplit& ts, void* scratch,
                  cudaStream_t s) {
  if (!scratch) return fail(CPC_ERR_WORKSPACE, "conv: the Chebyshev path needs its scratch");
  const int n = P->n;
  const SmoothScratch sm = smooth_scratch(P, ncols, scratch, sizeof(T));
  double* Part = sm.Part;
  ChebItem* recs = sm.recs;
  T* D = static_cast<T*>(sm.D);
  const void* tcheb = sizeof(T) == 4 ? static_cast<const void*>(P->d_tcheb32) : static_cast<const void*>(P->d_tcheb64);
  int slot = timing_begin("cheb_moments_kernel", s);
  cheb_moments_kernel<T><<<dim3((ncols + kChebCols - 1) / kChebCols, cheb_ranges(n)), kChebThreads, 0, s>>>(
      U, n, ncols, tcheb, Part);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("cheb_moments_kernel");
  const long long items = (long long)ncols * ts.n_smooth;
  slot = timing_begin("cheb_coef_kernel", s);
  cheb_coef_kernel<T><<<ncols, kChebCoefThreads, 0, s>>>(n, ncols, P->R_N, ts.smooth_q, ts.n_smooth,
                                                                 ts.smooth_k, P->d_cheb, Part, D, recs, sm.Mom,
                                                                 sm.Ddf);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("cheb_coef_kernel");
  slot = timing_begin("cheb_eval_kernel", s);
  auto kern = cheb_eval_kernel<T, DF>;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kChebThreads, 0));
  const int bx = std::max(1, n / (2 * kChebThreads));
  const long long by = std::max(1LL, std::min(items, ((long long)std::max(1, per_sm) * sm_count() + bx - 1) / bx));
  const void* te = DF ? static_cast<const void*>(P->d_tcheb32) : tcheb;
  const void* De = DF ? static_cast<const void*>(sm.Ddf) : static_cast<const void*>(D);
  kern<<<dim3(bx, unsigned(by)), kChebThreads, 0, s>>>(n, ncols, ts.n_smooth, te, De, recs, W);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("cheb_eval_kernel");
  return CPC_OK;
}

// all R_N terms of ncols columns: the banded and smooth terms from U (when
// given), the rest by FFT from the spectra or operands Uhat
template <typename T, bool SLICE, bool XIN>
int run_conv(const cpc_kernel* P, int ncols, const void* Uhat, void* W, const SliceOut& so, cudaStream_t s,
             const double* U, void* scratch) {
  if (ilog2(P->n) > kMaxLogN) return fail(CPC_ERR_UNSUPPORTED, "conv: n too large");
  if (SLICE && P->n < 128) return fail(CPC_ERR_UNSUPPORTED, "sliced conv: n must be at least 128");
  TermSplit ts = term_split(P, sizeof(T) == 4 ? 0 : 1, U);
  if (ts.n_smooth > 0 && !scratch) ts = term_split(P, sizeof(T) == 4 ? 0 : 1, nullptr);  // all by FFT
  int st = CPC_OK;
  if (ts.n_band > 0) {
    // (the sliced float32 form takes its lag-covered terms from the lag Gram
    // matrices: no slices for them)
    st = launch_band<T, SLICE>(P, ncols, U, static_cast<T*>(W), so, ts, s,
                               SLICE && sizeof(T) == 4 ? P->n_lag[0] : 0);
    if (st) return st;
  }
  if (ts.n_smooth > 0) {
    // (the sliced form's contraction takes these terms from their moments:
    // no slices)
    st = launch_smooth<T>(P, ncols, U, static_cast<T*>(W), ts, scratch, s);
    if (st) return st;
  }
  if (ts.n_fft > 0) st = dispatch_conv<T, kMinLogN, SLICE, XIN>(ilog2(P->n), P, ncols, Uhat, W, so, s, ts.fft_q, ts.n_fft);
  return st;
}

}  // namespace

template <int LOGN, int LOGP, typename V>
__global__ void pass_table_kernel(const V* __restrict__ flat, V* __restrict__ out,
                                  const double2* __restrict__ flat64, __half2* __restrict__ err) {
  constexpr int N = pass_table_size<LOGN, LOGP>();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const int e = pass_table_exponent<LOGN, LOGP>(k);
    out[k] = flat[e];
    if (err) {  // 2^24 (exact - float32) of each entry
      const double2 w = flat64[e];
      err[k] = __floats2half2_rn(float((w.x - double(flat[e].x)) * 16777216.0),
                                 float((w.y - double(flat[e].y)) * 16777216.0));
    }
  }
}

// the float32 operand factors of spectra32_kernel, per bin f < n:
// (1 + i e^{+i theta_f}, 1 - i e^{+i theta_f}), e^{-i theta_f} = hw64[f],
// formed in float64 and rounded once
__global__ void operand_factor_kernel(const double2* __restrict__ hw64, int n, float4* __restrict__ opf) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < n; f += gridDim.x * blockDim.x) {
    const double2 E = hw64[f];  // e^{-i theta}; e^{+i theta} = conj
    opf[f] = make_float4(float(1.0 + E.y), float(E.x), float(1.0 - E.y), float(-E.x));
  }
}

__global__ void error_table_kernel(const double2* __restrict__ w64, const float2* __restrict__ w32, int count,
                                   __half2* __restrict__ err) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x)
    err[k] = __floats2half2_rn(float((w64[k].x - double(w32[k].x)) * 16777216.0),
                               float((w64[k].y - double(w32[k].y)) * 16777216.0));
}

template <int LOGN>
int launch_pass_tables(cpc_kernel* P, cudaStream_t s) {
  constexpr int L64 = Geometry<LOGN, double>::LOGP, L32 = Geometry<LOGN, float>::LOGP;
  static_assert(pass_table_size<LOGN, L64>() <= (1 << LOGN) && pass_table_size<LOGN, L32>() <= (1 << LOGN),
                "pass tables fit in n entries");
  pass_table_kernel<LOGN, L64><<<8, 256, 0, s>>>(P->d_tw64, P->d_twp64, nullptr, nullptr);
  pass_table_kernel<LOGN, L32><<<8, 256, 0, s>>>(P->d_tw32, P->d_twp32, P->d_tw64,
                                                 static_cast<__half2*>(P->d_twp32_lo));
  error_table_kernel<<<8, 256, 0, s>>>(P->d_hw64, P->d_hw32, P->n + 1, static_cast<__half2*>(P->d_hw32_lo));
  operand_factor_kernel<<<8, 256, 0, s>>>(P->d_hw64, P->n, P->d_opf32);
  CPC_LAUNCH_CHECK("pass_table_kernel");
  return CPC_OK;
}

template <int LOGN>
int dispatch_pass_tables(int logn, cpc_kernel* P, cudaStream_t s) {
  if constexpr (LOGN > kMaxLogN) {
    return fail(CPC_ERR_UNSUPPORTED, "pass tables: n too large");
  } else {
    if (logn == LOGN) return launch_pass_tables<LOGN>(P, s);
    return dispatch_pass_tables<LOGN + 1>(logn, P, s);
  }
}

// per-pass twiddle tables of the float64 and float32 plans (n entries each,
// allocated by the caller), built from the flat tables
int build_pass_twiddles(cpc_kernel* P, cudaStream_t s) {
  return dispatch_pass_tables<kMinLogN>(ilog2(P->n), P, s);
}

int compute_kernel_spectrum(cpc_kernel* P, cudaStream_t s) {
  return dispatch_spectra<kMinLogN>(ilog2(P->n), 1, P->d_p, P->R_N, nullptr, nullptr, P->d_phat64,
                                    P->d_phat32, P, s);
}

int forward_spectra(const cpc_kernel* P, int ncols, const double* U, double2* Uhat64, float2* Uhat32,
                    cudaStream_t s) {
  return dispatch_spectra<kMinLogN>(ilog2(P->n), 0, U, ncols, Uhat64, Uhat32, nullptr, nullptr, P, s);
}

int forward_operands32(const cpc_kernel* P, int ncols, const double* U, void* X, cudaStream_t s) {
  return dispatch_spectra32<kMinLogN>(ilog2(P->n), U, ncols, static_cast<float4*>(X), P, s);
}

size_t operands32_bytes(const cpc_kernel* P, int ncols) { return align256(size_t(ncols) * P->n * sizeof(float4)); }

int build_kernel_pairs(cpc_kernel* P, cudaStream_t s) {
  kernel_pairs_kernel<<<64, 256, 0, s>>>(P->d_phat64, P->R_N, P->n, static_cast<float2*>(P->d_pp32));
  CPC_LAUNCH_CHECK("kernel_pairs_kernel");
  return CPC_OK;
}

// ---- host: the convolution path of every kernel term ----------------------
// Banded: from the float64 host tables p_q[m], m = 0..n-1 (the vector is
// even).  Class 0 (float32 W): the smallest H with the tail
// 2 sum_{m>H} |p_q[m]| at most 2^-32 of the whole sum
// |p_q[0]| + 2 sum_{m>0} |p_q[m]|, widened until the taps beyond (H+1)/2 hold
// at most 2^-9 of the sum (their lo parts are dropped); class 1 (float64 W):
// tail at most 2^-60 of the sum.  H is rounded up to an instantiated width.
static int band_half_width(const double* p, int n, int cls, std::vector<double>& tail) {
  const double tau = cls == 0 ? std::ldexp(1.0, -32) : std::ldexp(1.0, -60);
  double acc = 0.0;
  for (int m = n - 1; m >= 0; --m) {  // tail[H] = 2 sum_{m > H} |p[m]|
    tail[m] = acc;
    acc += (m > 0 ? 2.0 : 1.0) * std::fabs(p[m]);
  }
  const double sum = acc;
  if (!(sum > 0.0)) return -1;
  int H = 0;
  while (H < n - 1 && tail[H] > tau * sum) ++H;
  int need = H;
  if (cls == 0) {
    int L = 0;
    while (L < n - 1 && tail[L] > std::ldexp(sum, -9)) ++L;
    need = std::max(H, 2 * L - 1);
  }
  for (int k = 0; k < kBandNumWidths; ++k)
    if (band_width(k) >= need) return band_width(k) < n ? band_width(k) : -1;
  return -1;
}

// Smooth: the Chebyshev coefficients C[k][l] (k, l < kCheb) of
// g(x, y) = f_q(x - y) on [-b, b]^2, f_q(s) = a_q^{1/3} int_{s-h/2}^{s+h/2}
// exp(-t_q^2 x^2) dx (so f_q(m h) = p_q[m]), by interpolation at the
// kChebFit x kChebFit Chebyshev points of the first kind
// x_j = b cos(pi (j + 1/2) / kChebFit):
//   C[k][l] = (2 / N)^2 sum_{j,l'} g(x_j, x_l') T_k(x_j/b) T_l(x_l'/b),
// halved for k = 0 and for l = 0.
constexpr int kChebFit = 48;
static void cheb_fit(const cpc_kernel* P, int q, double* C) {
  constexpr int N = kChebFit;
  const double kPi = 3.14159265358979323846;
  const double b = P->b, h = P->h, t = P->t[q], sc = std::cbrt(P->a[q]);
  std::vector<double> x(N), A(size_t(kCheb) * N), g(size_t(N) * N), tmp(size_t(kCheb) * N);
  for (int j = 0; j < N; ++j) {
    const double th = kPi * (j + 0.5) / N;
    x[j] = b * std::cos(th);
    for (int k = 0; k < kCheb; ++k) A[size_t(k) * N + j] = (k == 0 ? 1.0 : 2.0) / N * std::cos(k * th);
  }
  for (int j = 0; j < N; ++j)
    for (int l = 0; l <= j; ++l) {
      const double d = x[j] - x[l];
      g[size_t(j) * N + l] = g[size_t(l) * N + j] = sc * gauss_cell_integral(t, d - 0.5 * h, d + 0.5 * h);
    }
  for (int k = 0; k < kCheb; ++k)
    for (int l = 0; l < N; ++l) {
      double acc = 0.0;
      for (int j = 0; j < N; ++j) acc += A[size_t(k) * N + j] * g[size_t(j) * N + l];
      tmp[size_t(k) * N + l] = acc;
    }
  for (int k = 0; k < kCheb; ++k)
    for (int m = 0; m < kCheb; ++m) {
      double acc = 0.0;
      for (int l = 0; l < N; ++l) acc += tmp[size_t(k) * N + l] * A[size_t(m) * N + l];
      C[size_t(k) * kCheb + m] = acc;
    }
}

// T_k(x_i / b) at the cell centres, k < kCheb: [kCheb][n]
static void cheb_table(int n, std::vector<double>& Tt) {
  Tt.resize(size_t(kCheb) * n);
  for (int i = 0; i < n; ++i) {
    const double th = std::acos(-1.0 + (2.0 * i + 1.0) / n);
    for (int k = 0; k < kCheb; ++k) Tt[size_t(k) * n + i] = std::cos(k * th);
  }
}

// The smallest rank K in {4, 8, 12, 16} (at most kmax) whose expansion
// matches p_q[|i - j|] within eps/4 of p_q[0] at a lattice of grid cells
// (97 indices per axis from 0 to n-1, all cells when n <= 97); -1 if none.
static int cheb_rank(const double* C, const double* p, const std::vector<double>& Tt, int n, int kmax, double eps) {
  std::vector<int> idx;
  if (n <= 97) {
    for (int i = 0; i < n; ++i) idx.push_back(i);
  } else {
    for (int m = 0; m <= 96; ++m) idx.push_back(int((long long)m * (n - 1) / 96));
  }
  const double bound = 0.25 * eps * std::fabs(p[0]);
  std::vector<double> V(idx.size() * kCheb);
  for (int K = 4; K <= std::min(kmax, kCheb); K += 4) {
    for (size_t jj = 0; jj < idx.size(); ++jj)
      for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int l = 0; l < K; ++l) acc += C[size_t(k) * kCheb + l] * Tt[size_t(l) * n + idx[jj]];
        V[jj * kCheb + k] = acc;
      }
    double err = 0.0;
    for (size_t ii = 0; ii < idx.size() && err <= bound; ++ii)
      for (size_t jj = 0; jj < idx.size(); ++jj) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += Tt[size_t(k) * n + idx[ii]] * V[jj * kCheb + k];
        err = std::max(err, std::fabs(acc - p[std::abs(idx[ii] - idx[jj])]));
      }
    if (err <= bound) return K;
  }
  return -1;
}

void plan_term_paths(const cpc_kernel* P, int band32, int band64, int rank32, int rank64, TermPlan& tp) {
  const int R_N = P->R_N, n = P->n;
  tp.terms.assign(size_t(2) * kTermRows * R_N, 0);
  tp.taps32.assign(size_t(R_N) * kBandTaps, make_float2(0.0f, 0.0f));
  tp.taps64.assign(size_t(R_N) * kBandTaps, 0.0);
  tp.cheb.assign(size_t(R_N) * kCheb * kCheb, 0.0);
  std::vector<double> tail(n);
  std::vector<char> fitted(R_N, 0);
  cheb_table(n, tp.tcheb);
  for (int cls = 0; cls < 2; ++cls) {
    const int hmax = cls == 0 ? band32 : band64;
    const int kmax = cls == 0 ? rank32 : rank64;
    const double eps = cls == 0 ? std::ldexp(1.0, -32) : std::ldexp(1.0, -44);
    int* hq = tp.terms.data() + size_t(cls) * kTermRows * R_N;
    int *kq = hq + R_N, *bl = hq + 2 * R_N, *sl = hq + 3 * R_N, *fl = hq + 4 * R_N, *dl = hq + 5 * R_N;
    int *cl = hq + 6 * R_N, *el = hq + 7 * R_N;
    int nb = 0, ns = 0, nf = 0;
    for (int q = 0; q < R_N; ++q) {
      const double* p = P->p.data() + size_t(q) * n;
      hq[q] = kq[q] = -1;
      const int H = hmax >= 0 ? band_half_width(p, n, cls, tail) : -1;
      if (H >= 0 && H <= hmax) {
        hq[q] = H;
        bl[nb++] = q;
        for (int m = 0; m <= H; ++m) {
          const float hi = float(p[m]);
          tp.taps32[size_t(q) * kBandTaps + m] = make_float2(hi, float(p[m] - double(hi)));
          tp.taps64[size_t(q) * kBandTaps + m] = p[m];
        }
        continue;
      }
      if (kmax >= 4 && p[0] > 0.0) {
        double* C = tp.cheb.data() + size_t(q) * kCheb * kCheb;
        if (!fitted[q]) {
          cheb_fit(P, q, C);
          fitted[q] = 1;
        }
        const int K = cheb_rank(C, p, tp.tcheb, n, kmax, eps);
        if (K > 0) {
          kq[q] = K;
          sl[ns++] = q;
          continue;
        }
      }
      fl[nf++] = q;
    }
    // the terms contracted over the cells: banded, then FFT
    for (int j = 0; j < nb; ++j) dl[j] = bl[j];
    for (int j = 0; j < nf; ++j) dl[nb + j] = fl[j];
    // tensor-core energy paths (FP32: class 0, FP64_TC: class 1): the banded
    // terms with H < L take their Gram matrices from the L lag Gram matrices
    // (L contractions instead of one per covered term); L minimises
    // L + (banded terms with H >= L), and the lag rows sit in the slice slots
    // of the first L covered terms
    int L = 0, cost = nb;
    for (int t = 1; t <= kMaxLags; ++t) {
        int cov = 0;
        for (int j = 0; j < nb; ++j) cov += hq[bl[j]] < t;
        if (cov >= t && t + (nb - cov) < cost) {
          cost = t + (nb - cov);
          L = t;
        }
      }
    int nc = 0, ne = 0;
    for (int j = 0; j < nb; ++j) {
      if (hq[bl[j]] < L) cl[nc++] = bl[j];
      else el[ne++] = bl[j];
    }
    for (int j = 0; j < nf; ++j) el[ne++] = fl[j];
    for (int m = 0; m < L; ++m) el[ne++] = cl[m];
    tp.n_band[cls] = nb;
    tp.n_smooth[cls] = ns;
    tp.n_lag[cls] = L;
    tp.n_cov[cls] = nc;
    tp.n_eh[cls] = ne;
  }
}

int build_term_tables(cpc_kernel* P, int band32, int band64, int rank32, int rank64, cudaStream_t s) {
  if (P->kind != CPC_KERNEL_CONV) return CPC_OK;
  const int R_N = P->R_N;
  TermPlan tp;
  plan_term_paths(P, band32, band64, rank32, rank64, tp);
  for (int cls = 0; cls < 2; ++cls) {
    const int* hq = tp.terms.data() + size_t(cls) * kTermRows * R_N;
    P->band_h[cls].assign(hq, hq + R_N);
    P->rank_k[cls].assign(hq + R_N, hq + 2 * R_N);
    P->n_band[cls] = tp.n_band[cls];
    P->n_smooth[cls] = tp.n_smooth[cls];
    P->n_lag[cls] = tp.n_lag[cls];
    P->n_cov[cls] = tp.n_cov[cls];
    P->n_eh[cls] = tp.n_eh[cls];
  }
  P->band_max[0] = band32;
  P->band_max[1] = band64;
  P->rank_max[0] = rank32;
  P->rank_max[1] = rank64;
  std::vector<float2> tc32(tp.tcheb.size());
  for (size_t k = 0; k < tp.tcheb.size(); ++k) {
    const float hi = float(tp.tcheb[k]);
    tc32[k] = make_float2(hi, float(tp.tcheb[k] - double(hi)));
  }
  if (!P->d_terms) {
    CPC_CUDA(cudaMalloc(&P->d_terms, sizeof(int) * tp.terms.size()));
    CPC_CUDA(cudaMalloc(&P->d_taps32, sizeof(float2) * tp.taps32.size()));
    CPC_CUDA(cudaMalloc(&P->d_taps64, sizeof(double) * tp.taps64.size()));
    CPC_CUDA(cudaMalloc(&P->d_cheb, sizeof(double) * tp.cheb.size()));
    CPC_CUDA(cudaMalloc(&P->d_tcheb32, sizeof(float2) * tc32.size()));
    CPC_CUDA(cudaMalloc(&P->d_tcheb64, sizeof(double) * tp.tcheb.size()));
  }
  CPC_CUDA(cudaMemcpyAsync(P->d_terms, tp.terms.data(), sizeof(int) * tp.terms.size(), cudaMemcpyHostToDevice, s));
  CPC_CUDA(cudaMemcpyAsync(P->d_taps32, tp.taps32.data(), sizeof(float2) * tp.taps32.size(), cudaMemcpyHostToDevice, s));
  CPC_CUDA(cudaMemcpyAsync(P->d_taps64, tp.taps64.data(), sizeof(double) * tp.taps64.size(), cudaMemcpyHostToDevice, s));
  CPC_CUDA(cudaMemcpyAsync(P->d_cheb, tp.cheb.data(), sizeof(double) * tp.cheb.size(), cudaMemcpyHostToDevice, s));
  CPC_CUDA(cudaMemcpyAsync(P->d_tcheb32, tc32.data(), sizeof(float2) * tc32.size(), cudaMemcpyHostToDevice, s));
  CPC_CUDA(cudaMemcpyAsync(P->d_tcheb64, tp.tcheb.data(), sizeof(double) * tp.tcheb.size(), cudaMemcpyHostToDevice, s));
  CPC_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  return CPC_OK;
}

int convolve_from_spectra(const cpc_kernel* P, int ncols, const void* Uhat, void* W, int precision,
                          cudaStream_t s, const double* U, void* scratch) {
  const SliceOut none{nullptr, 0, nullptr, 0};
  if (precision == CPC_FP64) return run_conv<double, false, false>(P, ncols, Uhat, W, none, s, U, scratch);
  return run_conv<float, false, false>(P, ncols, Uhat, W, none, s, U, scratch);
}

int convolve_operands32(const cpc_kernel* P, int ncols, const void* X, float* W, cudaStream_t s, const double* U,
                        void* scratch) {
  const SliceOut none{nullptr, 0, nullptr, 0};
  return run_conv<float, false, true>(P, ncols, X, W, none, s, U, scratch);
}

int convolve_operands32_sliced(const cpc_kernel* P, int R_f, const void* X, float* W, __nv_bfloat16* slices,
                               long long slice_stride, int* expo, cudaStream_t s, const double* U, void* scratch) {
  const SliceOut so{slices, slice_stride, expo, R_f};
  return run_conv<float, true, true>(P, 3 * R_f, X, W, so, s, U, scratch);
}

int convolve_spectra_df(const cpc_kernel* P, int ncols, void* Uhat, double* W, cudaStream_t s, const double* U,
                        void* scratch, const SliceRows* so64) {
  if (ilog2(P->n) > kMaxLogN) return fail(CPC_ERR_UNSUPPORTED, "conv: n too large");
  if (!P->d_twdf) return fail(CPC_ERR_INVALID, "conv: kernel has no double-float tables");
  if (so64 && !conv_slices64_supported(P)) return fail(CPC_ERR_UNSUPPORTED, "sliced float64 conv: n out of range");
  const SliceOut so = so64 ? *so64 : SliceOut{nullptr, 0, nullptr, 0};
  TermSplit ts = term_split(P, 1, U);
  if (ts.n_smooth > 0 && !scratch) ts = term_split(P, 1, nullptr);
  int st = CPC_OK;
  if (ts.n_band > 0) {
    // (FP64_TC: the lag-covered terms get no slices)
    st = so64 ? launch_band<double, true, true>(P, ncols, U, W, so, ts, s, P->n_lag[1])
              : launch_band<double, false, true>(P, ncols, U, W, so, ts, s);
    if (st) return st;
  }
  if (ts.n_smooth > 0) {
    st = launch_smooth<double, true>(P, ncols, U, W, ts, scratch, s);  // no slices (see run_conv)
    if (st) return st;
  }
  if (ts.n_fft > 0) {
    const dfc* X = static_cast<const dfc*>(Uhat);
    st = so64 ? dispatch_conv_df<kMinLogN, true>(ilog2(P->n), P, ncols, X, W, so, s, ts.fft_q, ts.n_fft)
              : dispatch_conv_df<kMinLogN, false>(ilog2(P->n), P, ncols, X, W, so, s, ts.fft_q, ts.n_fft);
  }
  return st;
}

// the float64 sliced convolution needs whole 128-cell tiles
bool conv_slices64_supported(const cpc_kernel* P) { return P->n >= 128 && P->n % 128 == 0; }

bool cheb_gram_active(const cpc_kernel* P, int cls) { return P->d_terms && P->n_smooth[cls] > 0; }

const int* dense_terms(const cpc_kernel* P, int cls, int* n_q) {
  if (!cheb_gram_active(P, cls)) {
    *n_q = P->R_N;
    return nullptr;
  }
  *n_q = P->R_N - P->n_smooth[cls];
  return P->d_terms + (size_t)cls * kTermRows * P->R_N + 5 * P->R_N;
}

const int* eh_terms(const cpc_kernel* P, int cls, int* n_q, int* n_virtual) {
  if (!P->d_terms || P->n_eh[cls] == 0 || (P->n_smooth[cls] == 0 && P->n_lag[cls] == 0)) {
    *n_q = P->R_N;
    *n_virtual = 0;
    return nullptr;
  }
  *n_q = P->n_eh[cls];
  *n_virtual = P->n_lag[cls];
  return P->d_terms + (size_t)cls * kTermRows * P->R_N + 7 * P->R_N;
}

int lag_slices64(const cpc_kernel* P, int R_f, const double* U, const SliceRows& so, cudaStream_t s) {
  const int L = P->n_lag[1];
  if (L == 0) return CPC_OK;
  const size_t smem = sizeof(double) * (size_t(P->n) + 2 * kMaxLags);
  int st = configure(lag_slice64_kernel, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lag_slice64_kernel, kLagThreads, smem));
  const long long grid = std::max(1LL, std::min(3LL * R_f, (long long)std::max(1, per_sm) * sm_count()));
  const int slot = timing_begin("lag_slice32_kernel", s);
  lag_slice64_kernel<<<unsigned(grid), kLagThreads, smem, s>>>(U, P->n, R_f, P->R_N, L,
                                                               P->d_terms + (size_t)kTermRows * P->R_N + 6 * P->R_N, so);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("lag_slice64_kernel");
  return CPC_OK;
}

int launch_lag_gram64(const cpc_kernel* P, int R_f, const double* S, double* G, cudaStream_t s) {
  const int L = P->n_lag[1];
  if (L == 0) return CPC_OK;
  const int nt = gram_tiles(R_f);
  const dim3 grid(unsigned(nt * (nt + 1) / 2), unsigned(P->n_cov[1]));
  const int* rows = P->d_terms + (size_t)kTermRows * P->R_N;
  const int slot = timing_begin("lag_gram_kernel", s);
  lag_gram64_kernel<<<grid, kGramThreads, 0, s>>>(R_f, P->R_N, L, rows + 6 * P->R_N, rows, P->d_taps64, S, G);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("lag_gram64_kernel");
  return CPC_OK;
}

int lag_slices32(const cpc_kernel* P, int R_f, const double* U, const SliceRows& so, cudaStream_t s) {
  const int L = P->n_lag[0];
  if (L == 0) return CPC_OK;
  const size_t smem = sizeof(float) * (size_t(P->n) + 2 * kMaxLags);
  int st = configure(lag_slice32_kernel, smem);
  if (st) return st;
  int per_sm = 0;
  CPC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lag_slice32_kernel, kLagThreads, smem));
  const long long grid = std::max(1LL, std::min(3LL * R_f, (long long)std::max(1, per_sm) * sm_count()));
  const int slot = timing_begin("lag_slice32_kernel", s);
  lag_slice32_kernel<<<unsigned(grid), kLagThreads, smem, s>>>(U, P->n, R_f, P->R_N, L, P->d_terms + 6 * P->R_N, so);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("lag_slice32_kernel");
  return CPC_OK;
}

size_t lag_gram_partials(const cpc_kernel* P, int R_f) {
  const size_t nt = gram_tiles(R_f);
  return size_t(P->R_N) * nt * (nt + 1) / 2;
}

int launch_lag_gram(const cpc_kernel* P, int R_f, const double* S, const double* c, double* G, double* partial,
                    long long* n_partial, cudaStream_t s) {
  *n_partial = 0;
  const int L = P->n_lag[0];
  if (L == 0) return CPC_OK;
  const int nt = gram_tiles(R_f);
  const dim3 grid(unsigned(nt * (nt + 1) / 2), unsigned(P->n_cov[0]));
  const int slot = timing_begin("lag_gram_kernel", s);
  lag_gram_kernel<<<grid, kGramThreads, 0, s>>>(R_f, P->R_N, L, P->d_terms + 6 * P->R_N, P->d_terms, P->d_taps32, S,
                                                c, G, partial);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("lag_gram_kernel");
  *n_partial = (long long)grid.x * grid.y;
  return CPC_OK;
}

size_t cheb_moment_rows_scratch(const cpc_kernel* P, int ncols) {
  return align256(sizeof(double) * size_t(cheb_ranges(P->n)) * ncols * kCheb);
}

int cheb_moment_rows(const cpc_kernel* P, int ncols, const double* U, void* Part, double* out, int width,
                     cudaStream_t s) {
  if (!P->d_tcheb32 || width < kCheb) return fail(CPC_ERR_INVALID, "cheb_moment_rows: no Chebyshev table");
  const int n = P->n;
  double* pt = static_cast<double*>(Part);
  int slot = timing_begin("cheb_moments_kernel", s);
  cheb_moments_kernel<float><<<dim3((ncols + kChebCols - 1) / kChebCols, cheb_ranges(n)), kChebThreads, 0, s>>>(
      U, n, ncols, P->d_tcheb32, pt);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("cheb_moments_kernel");
  const long long tot = (long long)ncols * width;
  moment_rows_kernel<<<unsigned((tot + 255) / 256), 256, 0, s>>>(pt, cheb_ranges(n), ncols, out, width);
  CPC_LAUNCH_CHECK("moment_rows_kernel");
  return CPC_OK;
}

int cheb_coef_rows(const cpc_kernel* P, int R_rho, const void* scratch, float* out, int width, cudaStream_t s) {
  if (!cheb_gram_active(P, 0) || width < kCheb) return fail(CPC_ERR_INVALID, "cheb_coef_rows: no smooth terms");
  const SmoothScratch sm = smooth_scratch(P, 3 * R_rho, scratch, sizeof(float));
  const long long rows = 3LL * R_rho * P->n_smooth[0];
  const long long tot = rows * width;
  coef_rows_kernel<<<unsigned((tot + 255) / 256), 256, 0, s>>>(static_cast<const float*>(sm.D), rows, out, width);
  CPC_LAUNCH_CHECK("coef_rows_kernel");
  return CPC_OK;
}

size_t cheb_gram_partials(const cpc_kernel* P, int R_f) {
  const size_t nt = gram_tiles(R_f);
  return size_t(P->R_N) * nt * (nt + 1) / 2;
}

int launch_cheb_gram(const cpc_kernel* P, int cls, int R_f, const void* scratch, const double* c, double* G,
                     double* partial, long long* n_partial, cudaStream_t s) {
  *n_partial = 0;
  if (!cheb_gram_active(P, cls)) return CPC_OK;
  const int ncols = 3 * R_f;
  const SmoothScratch sm = smooth_scratch(P, ncols, scratch, cls == 0 ? sizeof(float) : sizeof(double));
  const int R_N = P->R_N, n_smooth = P->n_smooth[cls];
  const int* rows = P->d_terms + (size_t)cls * kTermRows * R_N;  // K per term, then the smooth list
  const int nt = gram_tiles(R_f);
  const dim3 grid(unsigned(nt * (nt + 1) / 2), unsigned(n_smooth));
  const int slot = timing_begin("cheb_gram_kernel", s);
  cheb_gram_kernel<<<grid, kGramThreads, 0, s>>>(R_f, R_N, rows + 3 * R_N, n_smooth, rows + R_N, sm.Mom, sm.Ddf, c, G,
                                                 partial);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("cheb_gram_kernel");
  *n_partial = (long long)grid.x * grid.y;
  return CPC_OK;
}

int build_df_tables(cpc_kernel* P, cudaStream_t s) {
  const int n = P->n;
  CPC_CUDA(cudaMalloc(&P->d_twdf, sizeof(float4) * size_t(n)));
  CPC_CUDA(cudaMalloc(&P->d_hwdf, sizeof(float4) * size_t(n + 1)));
  CPC_CUDA(cudaMalloc(&P->d_phatdf, sizeof(float2) * size_t(P->R_N) * (n + 1)));
  to_df_copy_kernel<<<64, 256, 0, s>>>(reinterpret_cast<const double*>(P->d_twp64), reinterpret_cast<float2*>(P->d_twdf),
                                      2LL * n);
  to_df_copy_kernel<<<64, 256, 0, s>>>(reinterpret_cast<const double*>(P->d_hw64), reinterpret_cast<float2*>(P->d_hwdf),
                                      2LL * (n + 1));
  to_df_copy_kernel<<<64, 256, 0, s>>>(P->d_phat64, P->d_phatdf, (long long)P->R_N * (n + 1));
  CPC_LAUNCH_CHECK("to_df_copy_kernel");
  return CPC_OK;
}

size_t smooth_scratch_bytes(const cpc_kernel* P, int ncols) {
  // the layout of smooth_scratch (coefficients sized for float64 twice: the W
  // type's and the float64 copy)
  return align256(sizeof(double) * size_t(cheb_ranges(P->n)) * ncols * kCheb) +
         align256(sizeof(ChebItem) * size_t(ncols) * P->R_N) +
         2 * align256(sizeof(double) * size_t(ncols) * P->R_N * kCheb) + align256(sizeof(double) * size_t(ncols) * kCheb);
}

size_t spectra_bytes(const cpc_kernel* P, int ncols, int precision) {
  const size_t bins = size_t(ncols) * (P->n + 1);
  return align256(bins * (precision == CPC_FP64 ? sizeof(double2) : sizeof(float2)));
}

}  // namespace cpc

using namespace cpc;

namespace cpc {
// the spectra (or float32 operands) part of the convolution workspace; the
// Chebyshev scratch follows it
size_t conv_spectra_bytes(const cpc_kernel* P, int R_f, int precision) {
  precision = storage_precision(precision);
  // float32 forms keep a float64 copy of the spectra too (they are formed in float64)
  size_t b = spectra_bytes(P, 3 * R_f, precision);
  if (precision != CPC_FP64) b += spectra_bytes(P, 3 * R_f, CPC_FP64);
  return b;
}
}  // namespace cpc

extern "C" size_t cp_convolve_workspace(const cpc_kernel* P, int R_f, int precision) {
  if (!P || R_f <= 0) return 0;
  return conv_spectra_bytes(P, R_f, precision) + smooth_scratch_bytes(P, 3 * R_f);
}

namespace cpc {
// kernel kind, rank, factor pointers and precision (everything but the workspace)
int check_conv_inputs(const cpc_kernel* P, int R_f, const void* U, const void* W, int precision,
                      const char* who) {
  if (!P) return fail(CPC_ERR_INVALID, std::string(who) + ": NULL kernel");
  if (P->kind != CPC_KERNEL_CONV) return fail(CPC_ERR_INVALID, std::string(who) + ": needs a CONV kernel");
  if (R_f <= 0) return fail(CPC_ERR_INVALID, std::string(who) + ": R_f must be positive");
  if (!U || !W) return fail(CPC_ERR_INVALID, std::string(who) + ": NULL factor pointer");
  if ((reinterpret_cast<uintptr_t>(U) & 15) || (reinterpret_cast<uintptr_t>(W) & 15))
    return fail(CPC_ERR_INVALID, std::string(who) + ": U and W must be 16-byte aligned");
  if (!known_precision(precision))
    return fail(CPC_ERR_UNSUPPORTED, std::string(who) + ": precision form not implemented");
  return CPC_OK;
}

int check_conv_args(const cpc_kernel* P, int R_f, const void* U, const void* W, int precision,
                    void* ws, size_t ws_bytes, const char* who) {
  const int st = check_conv_inputs(P, R_f, U, W, precision, who);
  if (st) return st;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(CPC_ERR_WORKSPACE, std::string(who) + ": workspace NULL or not 256-byte aligned");
  if (ws_bytes < cp_convolve_workspace(P, R_f, precision))
    return fail(CPC_ERR_WORKSPACE, std::string(who) + ": workspace too small");
  return CPC_OK;
}

int run_convolve(const cpc_kernel* P, int R_f, const double* U, void* W, int precision, void* ws, cudaStream_t s,
                 const SliceRows* so64) {
  if (so64 && precision != CPC_FP64_TC) return fail(CPC_ERR_INVALID, "conv: W slices only for CPC_FP64_TC");
  const int ncols = 3 * R_f;
  // CPC_SPLIT and CPC_FP64_TC: FFT terms in double-float arithmetic
  const bool dfloat = precision == CPC_SPLIT || precision == CPC_FP64_TC;
  precision = storage_precision(precision);
  unsigned char* w = static_cast<unsigned char*>(ws);
  double2* h64 = reinterpret_cast<double2*>(w);
  int st;
  void* scratch = w + conv_spectra_bytes(P, R_f, precision);
  if (precision == CPC_FP64 && dfloat) {
    // factor spectra as double-float pairs in the float64-spectra part of the workspace
    st = dispatch_spectra_df<kMinLogN>(ilog2(P->n), U, ncols, reinterpret_cast<dfc*>(h64), P, s);
    if (st) return st;
    return convolve_spectra_df(P, ncols, h64, static_cast<double*>(W), s, U, scratch, so64);
  }
  if (precision == CPC_FP64) {
    st = forward_spectra(P, ncols, U, h64, nullptr, s);
    if (st) return st;
    return convolve_from_spectra(P, ncols, h64, W, precision, s, U, scratch);
  }
  // float32: the convolution operands straight from the float64 transforms
  // (they fit in the float64-spectra part of the workspace)
  st = forward_operands32(P, ncols, U, h64, s);
  if (st) return st;
  return convolve_operands32(P, ncols, h64, static_cast<float*>(W), s, U, scratch);
}
}  // namespace cpc

extern "C" int cp_convolve(const cpc_kernel* P, int R_f, const double* U, void* W, int precision,
                           void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  int st = check_conv_args(P, R_f, U, W, precision, ws, ws_bytes, "cp_convolve");
  if (st) return st;
  return run_convolve(P, R_f, U, W, precision, ws, static_cast<cudaStream_t>(stream));
}
