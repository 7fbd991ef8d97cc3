// Shared-memory Stockham FFT building blocks for sm_103a.
//
// A complex FFT of size NC = 2^LOGN is computed by NC/P threads, each holding
// P = 2^LOGP points in registers per pass.  The first pass has radix
// R1 = 2^(LOGN - (NP-1) LOGP) with B1 = P/R1 butterflies per thread, the other
// NP-1 passes have radix P.  Passes read and write one shared-memory buffer in
// place (all loads of a pass complete, a barrier, then all stores); the buffer
// index is padded by one element per 16 so the strided stores of the early
// passes do not collide in shared-memory banks.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "dfloat.cuh"

namespace cpc {

template <typename T> struct cvec;
template <> struct cvec<double> { using type = double2; };
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<df> { using type = dfc; };

// read-only loads of table entries (double-float entries as one 16-byte load)
__device__ __forceinline__ float2 ld_tw(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ld_tw(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dfc ld_tw(const dfc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  dfc r;
  r.x = df(v.x, v.y);
  r.y = df(v.z, v.w);
  return r;
}

template <typename V> __device__ __forceinline__ V cmk(decltype(V::x) x, decltype(V::x) y) { V r; r.x = x; r.y = y; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return cmk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
// multiply by SIGN * i
template <int SIGN, typename V> __device__ __forceinline__ V mul_si(V a) {
  return SIGN > 0 ? cmk<V>(-a.y, a.x) : cmk<V>(a.y, -a.x);
}

__host__ __device__ constexpr int pad_index(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }

// cos(2 pi j / 32), sin(2 pi j / 32), j = 0..7 (first octant; the rest by symmetry)
__device__ __forceinline__ double c32(int j) {
  const double t[9] = {1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708,
                       0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173,
                       0.19509032201612826785, 0.0};
  return t[j];
}

// exp(SIGN * 2 pi i k / R) for R | 32 and 0 <= k < R/2, built from the octant table.
template <typename V, int R, int SIGN>
__device__ __forceinline__ V root(int k) {
  using T = decltype(V::x);
  int j = k * (32 / R);  // angle 2 pi j / 32, j in [0, 16)
  double c, s;
  if (j <= 8) { c = c32(j); s = c32(8 - j); }          // [0, pi/2]
  else { c = -c32(16 - j); s = c32(j - 8); }            // (pi/2, pi)
  return cmk<V>(T(c), T(SIGN * s));
}

// float32 transforms carry each rounded constant's error as a second term
// (c = c_hi + c_lo): a handful of constants and table twiddles enter every
// transform, so without the second term their rounding errors do not average
// out and bias the result (about 1e-7 relative at n = 8192).

// x * (c + i s) for c, s known in double; float32: compensated
template <typename V>
__device__ __forceinline__ V cmul_const(V x, double c, double s) {
  using T = decltype(V::x);
  if constexpr (sizeof(T) == 4) {
    const float ch = float(c), sh = float(s);
    const float cl = float(c - double(ch)), sl = float(s - double(sh));
    const float re = fmaf(x.x, ch, fmaf(-x.y, sh, fmaf(x.x, cl, -x.y * sl)));
    const float im = fmaf(x.x, sh, fmaf(x.y, ch, fmaf(x.x, sl, x.y * cl)));
    return cmk<V>(re, im);
  } else {
    return cmul(x, cmk<V>(T(c), T(s)));
  }
}

// a / sqrt2 (float32: compensated)
template <typename T>
__device__ __forceinline__ T div_sqrt2(T a) {
  constexpr double r = 0.70710678118654752440;
  if constexpr (sizeof(T) == 4) {
    constexpr float rh = float(r), rl = float(r - double(float(r)));
    return fmaf(a, rh, a * rl);
  } else {
    return T(r) * a;
  }
}

// x * exp(SIGN 2 pi i k / R), with the trivial angles special-cased (k is a
// compile-time constant after unrolling, so the branches fold away).
template <typename V, int R, int SIGN>
__device__ __forceinline__ V rotate(V x, int k) {
  if (k == 0) return x;
  if (4 * k == R) return mul_si<SIGN>(x);
  if (8 * k == R) {  // (1 + SIGN i)/sqrt2
    return SIGN > 0 ? cmk<V>(div_sqrt2(x.x - x.y), div_sqrt2(x.x + x.y))
                    : cmk<V>(div_sqrt2(x.x + x.y), div_sqrt2(x.y - x.x));
  }
  if (8 * k == 3 * R) {  // (-1 + SIGN i)/sqrt2
    return SIGN > 0 ? cmk<V>(-div_sqrt2(x.x + x.y), div_sqrt2(x.x - x.y))
                    : cmk<V>(div_sqrt2(x.y - x.x), -div_sqrt2(x.x + x.y));
  }
  const int j = k * (32 / R);  // angle 2 pi j / 32, j in [0, 16)
  double c, s;
  if (j <= 8) { c = c32(j); s = c32(8 - j); }          // [0, pi/2]
  else { c = -c32(16 - j); s = c32(j - 8); }            // (pi/2, pi)
  return cmul_const(x, c, SIGN * s);
}

// In-register DFT of size R (power of two, R <= 32), unnormalised,
// X[k] = sum_j v[j] exp(SIGN 2 pi i j k / R); radix-2 decimation in time.
template <int R, int SIGN, typename V>
__device__ __forceinline__ void dft(V* v) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else {
    V e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    dft<R / 2, SIGN>(e);
    dft<R / 2, SIGN>(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      V t = rotate<V, R, SIGN>(o[k], k);
      v[k] = cadd(e[k], t);
      v[k + R / 2] = csub(e[k], t);
    }
  }
}

template <int LOGN, int LOGP>
struct FftPlan {
  static constexpr int NC = 1 << LOGN;
  static constexpr int P = 1 << LOGP;
  static constexpr int NP = (LOGN + LOGP - 1) / LOGP;  // number of passes
  static constexpr int LOGR1 = LOGN - (NP - 1) * LOGP;
  static constexpr int R1 = 1 << LOGR1;
  static constexpr int B1 = P / R1;
  static constexpr int TPF = NC / P;  // threads per FFT
  static_assert(LOGN >= LOGP, "FFT smaller than one thread's points");
};

// Twiddle: x * w^e for w = exp(-2 pi i / NC) (SIGN < 0) or its conjugate;
// `k` indexes the pass table (below), which holds w^e.  float32 tables come
// with a second table of the rounding errors, 2^24 (w^e - fl(w^e)) in fp16.
template <int SIGN, typename V>
__device__ __forceinline__ V twiddle(V x, const V* __restrict__ twp, const __half2* __restrict__ twl, int k) {
  V w = ld_tw(twp + k);
  if constexpr (sizeof(decltype(V::x)) == 4) {
    const float2 l = __half22float2(__ldg(twl + k));
    const float lx = l.x * (1.0f / 16777216.0f), ly = (SIGN > 0 ? -l.y : l.y) * (1.0f / 16777216.0f);
    const float wy = SIGN > 0 ? -w.y : w.y;
    const float re = fmaf(x.x, w.x, fmaf(-x.y, wy, fmaf(x.x, lx, -x.y * ly)));
    const float im = fmaf(x.x, wy, fmaf(x.y, w.x, fmaf(x.x, ly, x.y * lx)));
    return cmk<V>(re, im);
  } else {
    return SIGN > 0 ? cmulc(x, w) : cmul(x, w);
  }
}

// Pass tables.  Pass p >= 1 of a plan (Ns = R1 P^(p-1) butterfly groups,
// radix P) multiplies point r of butterfly j by w^((j mod Ns) (NC/(Ns P)) r).
// Its table stores these values at (r-1) Ns + (j mod Ns), so that the lanes
// of a warp (consecutive j) read consecutive entries; the tables of passes
// 1..NP-1 follow each other (offset of pass p: sum over earlier passes of
// (P-1) Ns).  The entries are copies of the flat table w^e, e = 0..NC-1.
template <int LOGN, int LOGP>
__host__ __device__ constexpr int pass_table_offset(int p) {
  using PL = FftPlan<LOGN, LOGP>;
  int off = 0, Ns = PL::R1;
  for (int q = 1; q < p; ++q) { off += (PL::P - 1) * Ns; Ns *= PL::P; }
  return off;
}
template <int LOGN, int LOGP>
__host__ __device__ constexpr int pass_table_size() {
  return pass_table_offset<LOGN, LOGP>(FftPlan<LOGN, LOGP>::NP);
}
// flat-table exponent of entry k of the pass tables (inverse of the layout above)
template <int LOGN, int LOGP>
__host__ __device__ inline int pass_table_exponent(int k) {
  using PL = FftPlan<LOGN, LOGP>;
  int Ns = PL::R1;
  for (int p = 1; p < PL::NP; ++p) {
    const int sz = (PL::P - 1) * Ns;
    if (k < sz) {
      const int r = k / Ns + 1, m = k % Ns;
      return m * (PL::NC / (Ns * PL::P)) * r;
    }
    k -= sz;
    Ns *= PL::P;
  }
  return 0;
}

// Load + twiddle + DFT of one pass from the padded shared buffer.
// Butterfly j of this thread: j = b * (NC / (R*B)) + t; points j + r NC/R.
// twp: this pass's table (unused when Ns == 1).
template <int NC, int R, int B, int SIGN, typename V>
__device__ __forceinline__ void pass_compute(const V* sbuf, V (&v)[B][R], int t, int Ns,
                                             const V* __restrict__ twp, const __half2* __restrict__ twl) {
  constexpr int stride = NC / R;
  constexpr int nbf = NC / (R * B);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = b * nbf + t;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b][r] = sbuf[pad_index(j + r * stride)];
    if (Ns > 1) {
      const int m = j & (Ns - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) v[b][r] = twiddle<SIGN>(v[b][r], twp, twl, (r - 1) * Ns + m);
    }
    dft<R, SIGN>(v[b]);
  }
}

// Stockham store of one pass: output index (j/Ns)*Ns*R + j%Ns + r*Ns.
template <int NC, int R, int B, typename V>
__device__ __forceinline__ void pass_store(V* sbuf, const V (&v)[B][R], int t, int Ns) {
  constexpr int nbf = NC / (R * B);
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = b * nbf + t;
    const int base = (j & ~(Ns - 1)) * R + (j & (Ns - 1));
#pragma unroll
    for (int r = 0; r < R; ++r) sbuf[pad_index(base + r * Ns)] = v[b][r];
  }
}

// Middle passes 2..NP-1 (radix P, one butterfly per thread): smem -> smem.
// Enter with the first pass stored; leave with pass NP-1 stored and synced.
// tw (twl): the plan's pass tables (float32: and their error tables); the
// last pass uses tw + pass_table_offset(NP-1).
template <int LOGN, int LOGP, int SIGN, typename V>
__device__ __forceinline__ void middle_passes(V* sbuf, int t, const V* __restrict__ tw,
                                              const __half2* __restrict__ twl) {
  using PL = FftPlan<LOGN, LOGP>;
  int Ns = PL::R1;
  const V* twp = tw;
  const __half2* twlp = twl;
#pragma unroll 1
  for (int p = 1; p < PL::NP - 1; ++p) {
    V v[1][PL::P];
    pass_compute<PL::NC, PL::P, 1, SIGN>(sbuf, v, t, Ns, twp, twlp);
    __syncthreads();
    pass_store<PL::NC, PL::P, 1>(sbuf, v, t, Ns);
    __syncthreads();
    twp += (PL::P - 1) * Ns;
    twlp += (PL::P - 1) * Ns;
    Ns *= PL::P;
  }
}

}  // namespace cpc
