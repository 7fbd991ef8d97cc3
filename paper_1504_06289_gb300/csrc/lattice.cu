// Assembled lattice sums of Newton potentials (Sec. 5.1, Eq. CoulombLatTensCan)
// and their evaluation on a tensor sub-grid.
//
//   assemble_kernel : S[l][q][i] = sum_k p~_q[i - e_l[k]]  (shift-and-window of
//                     the 2n master vectors onto the n-cell box; O(R L n)).
//   subgrid_kernel  : V[s1][s2][s3] = h^-3 sum_q S1[q][i1] S2[q][i2] S3[q][i3],
//                     one thread per s3, a block per 32 (s1, s2) pairs whose
//                     products S1*S2 sit in shared memory; q is streamed in
//                     chunks of 16.  The float32 form sums the (positive)
//                     terms with a compensated (Kahan) float32 sum.  Sub-grid
//                     indices outside [0, n) are clamped, never dereferenced.
//   subgrid_tc_kernel : the float32 form on the tensor cores when R_N <= 64:
//                     V[(s1,s2)][s3] is a product of a (s3 x q) matrix S3 and
//                     a (q x pairs) matrix S1 * S2 (the MMA's M runs over s3,
//                     so that stores are coalesced), each row split exactly
//                     into four bf16 integer slices under a per-row power of
//                     two (a published error-free splitting, the "Ozaki
//                     scheme"); the slice products are summed exactly in TMEM
//                     (every group sum over 64 q is an integer below 2^24) and
//                     folded into float32 once per output.  prep_kernel slices
//                     the S3 rows and gathers the S1, S2 sub-grid values once
//                     per call.
#include <cuda_bf16.h>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cuda_runtime.h>

#include "cpc_internal.h"
#include "pow2.cuh"
#include "umma.cuh"

namespace cpc {

constexpr int kMaxLattice = 256;   // charges per axis
constexpr int kMaxRN = 129;        // 2*64+1
constexpr int kPairsPerBlock = 32;

struct Edges {
  int count[3];
  int e[3 * kMaxLattice];
};

__global__ void assemble_kernel(int n, int R_N, const double* __restrict__ Pm, Edges ed,
                                double* __restrict__ S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y, l = blockIdx.z;
  if (i >= n) return;
  const double* row = Pm + (size_t)q * 2 * n + n;  // row[j] = p~_q[j], j in [-n, n)
  int base = 0;
  for (int a = 0; a < l; ++a) base += ed.count[a];
  double s = 0.0;
  for (int k = 0; k < ed.count[l]; ++k) s += row[i - ed.e[base + k]];
  S[((size_t)l * R_N + q) * n + i] = s;
}

constexpr int kQChunk = 16;
constexpr int kMaxRNPad = ((kMaxRN + kQChunk - 1) / kQChunk) * kQChunk;

__device__ __forceinline__ int clamp_index(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

template <typename TV>
__global__ void __launch_bounds__(512)
subgrid_kernel(int n, int R_N, int n_sub, const double* __restrict__ S, const int* __restrict__ sub,
               double inv_h3, TV* __restrict__ V) {
  // thread -> s3; block -> kPairsPerBlock consecutive (s1, s2) pairs, s2 fastest.
  // ab[pp][q] = S1[q][i1] * S2[q][i2] for the block's pairs, zero-padded in q,
  // formed in float64 and stored in the output's type (no per-term conversion).
  __shared__ TV ab[kPairsPerBlock][kMaxRNPad];
  const int s3 = threadIdx.x;
  const long long pair0 = (long long)blockIdx.x * kPairsPerBlock;
  const long long n_pairs = (long long)n_sub * n_sub;
  const int RNp = ((R_N + kQChunk - 1) / kQChunk) * kQChunk;
  for (int idx = threadIdx.x; idx < kPairsPerBlock * RNp; idx += blockDim.x) {
    const int pp = idx / RNp, q = idx % RNp;
    const long long pr = pair0 + pp;
    double v = 0.0;
    if (pr < n_pairs && q < R_N) {
      const int s1 = int(pr / n_sub), s2 = int(pr % n_sub);
      const int i1 = clamp_index(sub[s1], n), i2 = clamp_index(sub[n_sub + s2], n);
      v = S[(size_t)q * n + i1] * S[(size_t)(R_N + q) * n + i2];
    }
    ab[pp][q] = TV(v);
  }
  __syncthreads();
  if (s3 >= n_sub) return;
  const int i3 = clamp_index(sub[2 * n_sub + s3], n);
  const double* S3 = S + (size_t)2 * R_N * n + i3;
  if constexpr (sizeof(TV) == 8) {
    double acc[kPairsPerBlock];
#pragma unroll
    for (int pp = 0; pp < kPairsPerBlock; ++pp) acc[pp] = 0.0;
    for (int q0 = 0; q0 < RNp; q0 += kQChunk) {
      double c[kQChunk];
#pragma unroll
      for (int j = 0; j < kQChunk; ++j) c[j] = (q0 + j < R_N) ? S3[(size_t)(q0 + j) * n] : 0.0;
#pragma unroll
      for (int pp = 0; pp < kPairsPerBlock; ++pp)
#pragma unroll
        for (int j = 0; j < kQChunk; ++j) acc[pp] = fma(ab[pp][q0 + j], c[j], acc[pp]);
    }
#pragma unroll
    for (int pp = 0; pp < kPairsPerBlock; ++pp)
      if (pair0 + pp < n_pairs) V[(pair0 + pp) * n_sub + s3] = TV(acc[pp] * inv_h3);
  } else {
    // float32 products, Kahan-compensated float32 sum (all terms are positive)
    float acc[kPairsPerBlock], comp[kPairsPerBlock];
#pragma unroll
    for (int pp = 0; pp < kPairsPerBlock; ++pp) { acc[pp] = 0.0f; comp[pp] = 0.0f; }
    for (int q0 = 0; q0 < RNp; q0 += kQChunk) {
      float c[kQChunk];
#pragma unroll
      for (int j = 0; j < kQChunk; ++j) c[j] = (q0 + j < R_N) ? float(S3[(size_t)(q0 + j) * n]) : 0.0f;
#pragma unroll
      for (int pp = 0; pp < kPairsPerBlock; ++pp)
#pragma unroll
        for (int j = 0; j < kQChunk; ++j) {
          const float term = ab[pp][q0 + j] * c[j] - comp[pp];
          const float t = acc[pp] + term;
          comp[pp] = (t - acc[pp]) - term;
          acc[pp] = t;
        }
    }
#pragma unroll
    for (int pp = 0; pp < kPairsPerBlock; ++pp)
      if (pair0 + pp < n_pairs) V[(pair0 + pp) * n_sub + s3] = TV(float(double(acc[pp]) * inv_h3));
  }
}

// ---- tensor-core float32 form -------------------------------------------------
namespace lat {
// V[(s1,s2)][s3] as D = A B^T per sub-tile: A = the S3 rows of 128 sub-grid
// points s3 (the MMA's M, one TMEM lane each, so that a warp's 32 lanes hold
// 32 consecutive s3 and every store of a warp writes 128 contiguous bytes),
// B = the products a_q = S1[q][i1] S2[q][i2] of 64 (s1, s2) pairs (the MMA's N).
constexpr int BM = 128;      // s3 points per sub-tile (TMEM lanes)
constexpr int NP = 64;       // (s1, s2) pairs per CTA (TMEM columns per slice group)
constexpr int NSL = 4;       // slices: x = 2^e (s0 2^-8 + s1 2^-16 + s2 2^-24 + s3 2^-32)
constexpr int THREADS = 256;        // 8 warps: lane quadrant x column half of the accumulators
constexpr int PREP_THREADS = BM;    // one S3 row per thread
constexpr uint32_t A_SLICE = BM * 128, B_SLICE = NP * 128;  // rows of 64 bf16 (128 bytes)
constexpr uint32_t TMEM_COLS = NSL * NP;                    // 256
constexpr long kSpinLimit = 20000000;
constexpr int kMaxSub = 512;
constexpr int kMaxTiles = kMaxSub / BM;
constexpr size_t kATileBytes = size_t(NSL) * A_SLICE;  // 64 KB per sub-tile
constexpr size_t kSmemBytes = kATileBytes + size_t(NSL) * B_SLICE + 1024 + 64 + 2 * NP * sizeof(int);
// per-call scratch of the MASTER kernel: the S3 rows sliced per sub-tile, their
// exponents, and the S1, S2 values of the sub-grid gathered q-contiguous
constexpr size_t kExpOff = kMaxTiles * kATileBytes;
constexpr size_t kGathOff = kExpOff + kMaxSub * sizeof(int);
constexpr size_t kScratchBytes = kGathOff + size_t(2) * kMaxSub * 64 * sizeof(double);

// NCH 16-byte chunks (8 values each, chunks c0 .. c0+NCH-1 of a 64-value row)
// -> NSL bf16 slices under the row exponent e (|x| < 2^e), written into
// 128-byte-swizzled K-major rows at `base` (slice k at base + k * slice_bytes)
template <int NCH>
__device__ __forceinline__ void slice_chunks(const float* x, int e, uint8_t* base, uint32_t slice_bytes, int row,
                                             int c0) {
  // x 2^(8-e) by one exact multiplication while 2^(8-e) is a normal float
  const bool fast = e > -100 && e < 100;
  const float sc = fast ? pow2f(8 - e) : 0.0f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    uint32_t w[NSL][4];
#pragma unroll
    for (int h = 0; h < 8; h += 2) {
      float sl[NSL][2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float a = fast ? x[8 * c + h + u] * sc : ldexpf(x[8 * c + h + u], 8 - e);  // |a| < 256
#pragma unroll
        for (int k = 0; k < NSL; ++k) {
          const float r = rintf(a);
          sl[k][u] = r;
          a = (a - r) * 256.0f;  // exact
        }
      }
#pragma unroll
      for (int k = 0; k < NSL; ++k) {
        const __nv_bfloat162 b2 = __floats2bfloat162_rn(sl[k][0], sl[k][1]);
        w[k][h / 2] = *reinterpret_cast<const uint32_t*>(&b2);
      }
    }
    const uint32_t off = umma::sw128_offset(row, (c0 + c) * 16);
#pragma unroll
    for (int k = 0; k < NSL; ++k)
      *reinterpret_cast<uint4*>(base + k * slice_bytes + off) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
  }
}

__device__ __forceinline__ int row_exponent(float m) {
  int e = 0;
  if (m > 0.0f) frexpf(m, &e);  // m < 2^e
  return e;
}

// Once per call.  blockIdx.y == 0: the S3 rows of sub-tile blockIdx.x sliced
// into the scratch (tile j at j * 64 KB, slice k at + k * 16 KB) with their
// exponents; blockIdx.y == 1, 2: the S1 (S2) values of the tile's sub-grid
// points gathered as rows g[s][q] (float64, zero for q >= R_N).
__global__ void __launch_bounds__(PREP_THREADS)
prep_kernel(int n, int R_N, int n_sub, const double* __restrict__ S, const int* __restrict__ sub,
            unsigned char* __restrict__ scratch) {
  const int t = threadIdx.x, j = blockIdx.x;
  if (blockIdx.y == 0) {
    const int s3 = j * BM + t;  // < kMaxSub
    const bool ok = s3 < n_sub;
    const int i3 = clamp_index(sub[2 * n_sub + (ok ? s3 : 0)], n);
    float x[64];
    float m = 0.0f;
#pragma unroll
    for (int q = 0; q < 64; ++q) {
      x[q] = (ok && q < R_N) ? float(S[(size_t)(2 * R_N + q) * n + i3]) : 0.0f;
      m = fmaxf(m, fabsf(x[q]));
    }
    const int e = row_exponent(m);
    slice_chunks<8>(x, e, scratch + (size_t)j * kATileBytes, A_SLICE, t, 0);
    reinterpret_cast<int*>(scratch + kExpOff)[s3] = ok ? e : 0;
  } else {
    const int l = blockIdx.y - 1;
    double* g = reinterpret_cast<double*>(scratch + kGathOff) + (size_t)l * kMaxSub * 64;
    for (int idx = t; idx < BM * 64; idx += PREP_THREADS) {
      const int s = j * BM + idx / 64, q = idx % 64;
      double v = 0.0;
      if (s < n_sub && q < R_N) v = S[(size_t)(l * R_N + q) * n + clamp_index(sub[l * n_sub + s], n)];
      g[(size_t)s * 64 + q] = v;
    }
  }
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void load_tile(uint32_t dst, const unsigned char* scratch, int j, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(umma::smem_u32(bar)),
               "r"(uint32_t(kATileBytes))
               : "memory");
  bulk_load(dst, scratch + (size_t)j * kATileBytes, uint32_t(kATileBytes), umma::smem_u32(bar));
}

// One CTA per 64 consecutive (s1, s2) pairs; it slices their products into
// shared memory once, then walks the sub-tiles of 128 s3 points: the tile's
// S3 slices arrive by one bulk copy (the next one during the fold), one thread
// issues the 10 slice-pair products per 16-q step, and eight warps (TMEM lane
// quadrant x half of the 64 columns) fold the four TMEM groups into float32
// and store V[(s1,s2)][s3].
__global__ void __launch_bounds__(THREADS, 2)
subgrid_tc_kernel(int n_sub, float inv_h3, const unsigned char* __restrict__ scratch, float* __restrict__ V) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = umma::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t* smem = smem_raw + pad;
  const uint32_t sA = raw + pad, sB = sA + uint32_t(kATileBytes);
  uint8_t* smemB = smem + kATileBytes;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kATileBytes + NSL * B_SLICE);  // MMAs done
  uint64_t* abar = mbar + 1;                                                          // S3 tile landed
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(abar + 1);
  int* eP = reinterpret_cast<int*>(smem + kATileBytes + NSL * B_SLICE + 64);  // exponents of the pair rows
  float* fP = reinterpret_cast<float*>(eP + NP);  // 2^eP, or 0 outside the fast range
  const int* eS = reinterpret_cast<const int*>(scratch + kExpOff);
  const double* g1 = reinterpret_cast<const double*>(scratch + kGathOff);
  const double* g2 = g1 + (size_t)kMaxSub * 64;

  const int t = threadIdx.x, warp = t >> 5;
  const long long n_pairs = (long long)n_sub * n_sub;
  const long long pair0 = (long long)blockIdx.x * NP;
  const int n_tiles = (n_sub + BM - 1) / BM;
  if (t == 0) {
    umma::mbar_init(mbar, 1);
    umma::mbar_init(abar, 1);
    umma::mbar_fence_init();
  }
  __syncthreads();
  if (t == 0) load_tile(sA, scratch, 0, abar);  // lands while the pair rows are formed
  {
    // pair row k = t / 4, quarter h = t % 4 (q = 16 h .. 16 h + 15):
    // a_q = S1[q][i1] S2[q][i2] (float64 product, rounded once)
    const int k = t >> 2, h = t & 3;
    const long long p = pair0 + k;
    const bool ok = p < n_pairs;
    const int s1 = ok ? int(p / n_sub) : 0, s2 = ok ? int(p % n_sub) : 0;
    const double2* r1 = reinterpret_cast<const double2*>(g1 + (size_t)s1 * 64 + 16 * h);
    const double2* r2 = reinterpret_cast<const double2*>(g2 + (size_t)s2 * 64 + 16 * h);
    float x[16];
    float m = 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double2 a = __ldg(r1 + u), b = __ldg(r2 + u);
      x[2 * u] = ok ? float(a.x * b.x) : 0.0f;
      x[2 * u + 1] = ok ? float(a.y * b.y) : 0.0f;
      m = fmaxf(m, fmaxf(fabsf(x[2 * u]), fabsf(x[2 * u + 1])));
    }
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));  // the row's other quarters
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    const int e = row_exponent(m);
    slice_chunks<2>(x, e, smemB, B_SLICE, k, 2 * h);
    if (h == 0) {
      eP[k] = e;
      fP[k] = (e > -100 && e < 100) ? pow2f(e) : 0.0f;
    }
  }
  if (warp == 0) umma::tmem_alloc(tmem_ptr, TMEM_COLS);
  umma::fence_proxy_async();  // the B slices (generic-proxy writes) -> tensor-core reads
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tbase = *tmem_ptr;
  const int quad = warp & 3, half = warp >> 2;  // TMEM lanes 32 quad.., columns 32 half..
  const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * quad) << 16) + half * (NP / 2);
  constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, NP);
  bool ok_wait = true;
  for (int j = 0; j < n_tiles; ++j) {
    ok_wait = ok_wait && umma::mbar_wait(abar, j & 1, kSpinLimit);
    if (t == 0) {
      umma::fence_after();
      // group g accumulates the slice pairs (a, b) with a + b = g
#pragma unroll
      for (int g = 0; g < NSL; ++g) {
        uint32_t acc = 0;
#pragma unroll
        for (int a = 0; a <= g; ++a) {
          const int b = g - a;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            umma::mma_bf16(tbase + g * NP, umma::desc_k_sw128(sA + a * A_SLICE + kk * 32),
                           umma::desc_k_sw128(sB + b * B_SLICE + kk * 32), idesc, acc);
            acc = 1;
          }
        }
      }
      umma::mma_commit(mbar);
    }
    ok_wait = ok_wait && umma::mbar_wait(mbar, j & 1, kSpinLimit);
    umma::fence_after();
    __syncthreads();  // every thread has passed its wait on this phase of abar
    // the MMAs have read this tile's S3 slices: the next tile's come during the fold
    if (t == 0 && j + 1 < n_tiles && ok_wait) load_tile(sA, scratch, j + 1, abar);
    // fold: v = (S0 + S1 2^-8 + S2 2^-16 + S3 2^-24) 2^(e3 + ep - 16) h^-3, the
    // power of two applied as two exact multiplications in the normal range
    const int s3 = j * BM + 32 * quad + (t & 31);
    const bool s_ok = s3 < n_sub;
    const int e3 = s_ok ? __ldg(eS + s3) : 0;
    const bool fast3 = e3 > -100 && e3 < 100;
    const float f3 = ldexpf(inv_h3, e3 - 16);
    // this warp's 32 pairs start at prow0; every store of a warp writes 32
    // consecutive s3 of one pair
    const long long prow0 = pair0 + half * (NP / 2);
    const bool full = prow0 + NP / 2 <= n_pairs;
    float* vrow = V + prow0 * n_sub + s3;
#pragma unroll
    for (int cb = 0; cb < NP / 16; ++cb) {
      float v0[8], v1[8], v2[8], v3[8];
      umma::tmem_ld8(lane_base + cb * 8, v0);
      umma::tmem_ld8(lane_base + NP + cb * 8, v1);
      umma::tmem_ld8(lane_base + 2 * NP + cb * 8, v2);
      umma::tmem_ld8(lane_base + 3 * NP + cb * 8, v3);
      umma::tmem_ld_wait();
      if (s_ok) {
        const int kb = half * (NP / 2) + cb * 8;
        const float4 fa = *reinterpret_cast<const float4*>(fP + kb);
        const float4 fb = *reinterpret_cast<const float4*>(fP + kb + 4);
        const float fpv[8] = {fa.x, fa.y, fa.z, fa.w, fb.x, fb.y, fb.z, fb.w};
        bool fast = fast3;
#pragma unroll
        for (int u = 0; u < 8; ++u) fast = fast && fpv[u] != 0.0f;
        float val[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          val[u] = fmaf(v3[u], 1.0f / 16777216.0f, fmaf(v2[u], 1.0f / 65536.0f, fmaf(v1[u], 1.0f / 256.0f, v0[u])));
        if (fast) {
#pragma unroll
          for (int u = 0; u < 8; ++u) val[u] = (val[u] * fpv[u]) * f3;
        } else {
          for (int u = 0; u < 8; ++u) val[u] = ldexpf(val[u], e3 + eP[kb + u] - 16) * inv_h3;
        }
        if (!ok_wait)
#pragma unroll
          for (int u = 0; u < 8; ++u) val[u] = __int_as_float(0x7fc00000);
        float* vp = vrow + (size_t)(cb * 8) * n_sub;
        if (full) {
#pragma unroll
          for (int u = 0; u < 8; ++u) __stcs(vp + u * n_sub, val[u]);
        } else {
          for (int u = 0; u < 8; ++u)
            if (prow0 + cb * 8 + u < n_pairs) __stcs(vp + u * n_sub, val[u]);
        }
      }
    }
    umma::fence_before();
    __syncthreads();  // TMEM is rewritten by the next tile's MMAs
    umma::fence_after();
  }
  if (warp == 0) umma::tmem_dealloc(tbase, TMEM_COLS);
}
}  // namespace lat

// the MASTER kernel's scratch: the sub-grid evaluation's (above), or the
// interaction energy's [3][R_N] axis sums (and list lengths) in the first
// 4 KB, then per axis a histogram of 2n bins and a list of up to 2n
// (d, count) pairs, whichever is larger
constexpr size_t kEnergyListOff = 4096;
size_t lattice_scratch_bytes(int n) {
  return std::max(lat::kScratchBytes, kEnergyListOff + size_t(3) * 2 * n * 3 * sizeof(int));
}

// ---- nuclear potential by windowed shifts of the master kernel (Sec. 3.3) ----
// F[l][a R_N + q][i] = p~_q[i - e[l][a]], i = 0..n-1: the master vector of
// term q shifted onto nucleus a (at the grid-cell edge e[l][a] of axis l) and
// windowed onto the n-cell box; float64, or rounded to float32.
template <typename T>
__global__ void window_kernel(int n, int R_N, int n_nuc, const double* __restrict__ Pm, Edges ed,
                              T* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y, l = blockIdx.z;
  if (i >= n) return;
  const int a = row / R_N, q = row - a * R_N;
  const int e = ed.e[l * n_nuc + a];  // in [0, n]: i - e in [-n, n-1]
  F[((size_t)l * n_nuc * R_N + row) * n + i] = T(Pm[(size_t)q * 2 * n + n + i - e]);
}

int launch_window(const cpc_kernel* P, int n_nuc, const int* edges, void* F, bool fp32, cudaStream_t s) {
  if (n_nuc < 1 || n_nuc > kMaxLattice) return fail(CPC_ERR_UNSUPPORTED, "nuclear factors: 1..256 nuclei");
  if ((long long)n_nuc * P->R_N > 65535) return fail(CPC_ERR_UNSUPPORTED, "nuclear factors: too many columns");
  Edges ed;
  for (int l = 0; l < 3; ++l) {
    ed.count[l] = n_nuc;
    for (int a = 0; a < n_nuc; ++a) {
      const int e = edges[l * n_nuc + a];
      if (e < 0 || e > P->n) return fail(CPC_ERR_INVALID, "nuclear factors: edge index outside [0, n]");
      ed.e[l * n_nuc + a] = e;
    }
  }
  const dim3 grid((P->n + 255) / 256, n_nuc * P->R_N, 3);
  if (fp32) window_kernel<float><<<grid, 256, 0, s>>>(P->n, P->R_N, n_nuc, P->d_p, ed, static_cast<float*>(F));
  else window_kernel<double><<<grid, 256, 0, s>>>(P->n, P->R_N, n_nuc, P->d_p, ed, static_cast<double*>(F));
  CPC_LAUNCH_CHECK("window_kernel");
  return CPC_OK;
}

// ---- interaction energy of the lattice charges (Sec. 5.3, Eq. EnergyLattice) ----
// A charge sits at the grid-cell edge e, the corner of the cells e-1 and e of
// each axis; the potential sum traced at a lattice point is the mean of those
// 8 cells (the doubled lattice of the traced 2L sub-tensor).  Per axis,
//   T_q = 1/2 sum_{j,k} (p~_q[e_j - e_k - 1] + p~_q[e_j - e_k])
//       = 1/2 sum_d c(d) (p~_q[d - 1] + p~_q[d]),
// c(d) the number of point pairs of the axis at difference d, the same for
// every q.  lattice_pairs_kernel counts the pairs of one slice of the L^2 in a
// shared-memory histogram over the 2n possible d and adds its nonzero bins to
// the axis histogram; lattice_diffs_kernel lists the nonzero bins in order of
// d; lattice_energy_kernel (block q, l) sums over that list.  A regular
// lattice of L points has 2L-1 differences, so the work per q is O(L).
constexpr int kPairChunks = 32;
constexpr int kPairThreads = 1024;
constexpr int kEnergyThreads = 128;

__global__ void __launch_bounds__(kPairThreads)
lattice_pairs_kernel(int n, Edges ed, int* __restrict__ ghist) {
  extern __shared__ int hist[];  // [2n]: c(d) at d + n
  __shared__ int se[kMaxLattice];
  const int c = blockIdx.x, l = blockIdx.y, t = threadIdx.x, nb = 2 * n;
  int base = 0;
  for (int a = 0; a < l; ++a) base += ed.count[a];
  const int L = ed.count[l];
  const int pairs = L * L, chunk = (pairs + kPairChunks - 1) / kPairChunks;
  const int p0 = c * chunk, p1 = min(pairs, p0 + chunk);
  if (p0 >= p1) return;  // nothing in this slice (uniform over the block)
  for (int i = t; i < nb; i += kPairThreads) hist[i] = 0;
  for (int i = t; i < L; i += kPairThreads) se[i] = ed.e[base + i];
  __syncthreads();
  for (int p = p0 + t; p < p1; p += kPairThreads)
    atomicAdd(&hist[se[p / L] - se[p % L] + n], 1);  // d + n in [2, 2n-2]
  __syncthreads();
  int* gh = ghist + (size_t)l * nb;
  for (int i = t; i < nb; i += kPairThreads)
    if (hist[i]) atomicAdd(&gh[i], hist[i]);
}

// the nonzero bins of axis blockIdx.x in order of d, as pairs (d, c(d)):
// chunks of 1024 consecutive bins (coalesced), each thread's position from a
// warp ballot and a block scan of the warp counts
__global__ void __launch_bounds__(kPairThreads)
lattice_diffs_kernel(int n, const int* __restrict__ ghist, int* __restrict__ list, int* __restrict__ list_len) {
  __shared__ int wcount[kPairThreads / 32];
  __shared__ int woff[kPairThreads / 32 + 1];
  const int l = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nb = 2 * n;
  const int* gh = ghist + (size_t)l * nb;
  int* out = list + (size_t)l * 2 * nb;  // up to 2n pairs
  int base = 0;
  for (int c0 = 0; c0 < nb; c0 += kPairThreads) {
    const int i = c0 + t;
    const int v = (i < nb) ? gh[i] : 0;
    const unsigned ball = __ballot_sync(0xffffffffu, v != 0);
    if (lane == 0) wcount[warp] = __popc(ball);
    __syncthreads();
    if (t == 0) {
      int acc = 0;
      for (int w = 0; w < kPairThreads / 32; ++w) {
        woff[w] = acc;
        acc += wcount[w];
      }
      woff[kPairThreads / 32] = acc;
    }
    __syncthreads();
    if (v) {
      const int pos = base + woff[warp] + __popc(ball & ((1u << lane) - 1u));
      out[2 * pos] = i - n;
      out[2 * pos + 1] = v;
    }
    base += woff[kPairThreads / 32];
    __syncthreads();  // wcount and woff are rewritten by the next chunk
  }
  if (t == 0) list_len[l] = base;
}

__global__ void __launch_bounds__(kEnergyThreads)
lattice_energy_kernel(int n, int R_N, const double* __restrict__ Pm, const int* __restrict__ list,
                      const int* __restrict__ list_len, double* __restrict__ T) {
  __shared__ double red[kEnergyThreads / 32];
  const int q = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
  const double* row = Pm + (size_t)q * 2 * n + n;  // row[j] = p~_q[j], j in [-n, n)
  const int* dl = list + (size_t)l * 4 * n;
  const int len = list_len[l];
  double s = 0.0;
  for (int i = t; i < len; i += kEnergyThreads) {
    const int d = dl[2 * i];  // in [-(n-2), n-2]
    s = fma(double(dl[2 * i + 1]), row[d - 1] + row[d], s);
  }
  // fixed-order reduction: the same sum on every call
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  if (t == 0) {
    double tot = 0.0;
    for (int w = 0; w < kEnergyThreads / 32; ++w) tot += red[w];
    T[(size_t)l * R_N + q] = 0.5 * tot;
  }
}

// E_L = Z^2 h^-3 / 2 sum_q (prod_l T[l][q] - L1 L2 L3 t0_q^3): the terms in
// parallel, their sum in order of q; products and the difference rounded
// separately (no fused multiply-add), so that a single charge gives exactly 0
__global__ void lattice_energy_sum_kernel(int n, int R_N, const double* __restrict__ Pm, const double* __restrict__ T,
                                          double count, double scale, double* __restrict__ E) {
  __shared__ double term[kMaxRN];
  for (int q = threadIdx.x; q < R_N; q += blockDim.x) {
    const double* row = Pm + (size_t)q * 2 * n + n;
    const double t0 = 0.5 * (row[-1] + row[0]);
    const double lat = __dmul_rn(__dmul_rn(T[q], T[R_N + q]), T[2 * R_N + q]);
    const double self = __dmul_rn(count, __dmul_rn(__dmul_rn(t0, t0), t0));
    term[q] = __dsub_rn(lat, self);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < R_N; ++q) s = __dadd_rn(s, term[q]);
    *E = __dmul_rn(scale, s);
  }
}

template <typename TV>
int launch_subgrid(int n, int R_N, int n_sub, const double* S, const int* sub, double inv_h3, void* V,
                   cudaStream_t s) {
  const long long n_pairs = (long long)n_sub * n_sub;
  const long long blocks = (n_pairs + kPairsPerBlock - 1) / kPairsPerBlock;
  const int threads = ((n_sub + 31) / 32) * 32;
  subgrid_kernel<TV><<<(unsigned)blocks, threads, 0, s>>>(n, R_N, n_sub, S, sub, inv_h3, static_cast<TV*>(V));
  CPC_LAUNCH_CHECK("subgrid_kernel");
  return CPC_OK;
}

}  // namespace cpc

using namespace cpc;

extern "C" int lattice_potential_sum(const cpc_kernel* P, const int* L, const int* edges, double* S, int n_sub,
                                     const int* sub, void* V, int precision, void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_MASTER) return fail(CPC_ERR_INVALID, "lattice_potential_sum: needs a MASTER kernel");
  if (!L || !edges || !S) return fail(CPC_ERR_INVALID, "lattice_potential_sum: NULL argument");
  const int n = P->n;
  Edges ed;
  int total = 0;
  for (int l = 0; l < 3; ++l) {
    if (L[l] < 0 || L[l] > kMaxLattice) return fail(CPC_ERR_UNSUPPORTED, "lattice_potential_sum: L per axis must be in [0, 256]");
    ed.count[l] = L[l];
    for (int k = 0; k < L[l]; ++k) {
      const int e = edges[total + k];
      if (e < 0 || e > n) return fail(CPC_ERR_INVALID, "lattice_potential_sum: edge index outside [0, n]");
      ed.e[total + k] = e;
    }
    total += L[l];
  }
  if (V) {
    if (n_sub <= 0 || n_sub > 512 || !sub) return fail(CPC_ERR_INVALID, "lattice_potential_sum: n_sub must be in [1, 512] with sub given");
    if (precision != CPC_FP64 && precision != CPC_FP32)
      return fail(CPC_ERR_UNSUPPORTED, "lattice_potential_sum: precision form not implemented");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dim3 grid((n + 255) / 256, P->R_N, 3);
  assemble_kernel<<<grid, 256, 0, s>>>(n, P->R_N, P->d_p, ed, S);
  CPC_LAUNCH_CHECK("assemble_kernel");
  if (!V) return CPC_OK;
  const double inv_h3 = 1.0 / (P->h * P->h * P->h);
  if (precision == CPC_FP64) return launch_subgrid<double>(n, P->R_N, n_sub, S, sub, inv_h3, V, s);
  if (P->R_N <= 64) {  // tensor cores
    const long long blocks = ((long long)n_sub * n_sub + lat::NP - 1) / lat::NP;
    CPC_CUDA(cudaFuncSetAttribute(lat::subgrid_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(lat::kSmemBytes)));
    lat::prep_kernel<<<dim3((n_sub + lat::BM - 1) / lat::BM, 3), lat::PREP_THREADS, 0, s>>>(n, P->R_N, n_sub, S, sub,
                                                                                     P->d_lat);
    CPC_LAUNCH_CHECK("lattice prep_kernel");
    const int slot = timing_begin("subgrid_tc_kernel", s);
    lat::subgrid_tc_kernel<<<(unsigned)blocks, lat::THREADS, lat::kSmemBytes, s>>>(n_sub, float(inv_h3), P->d_lat,
                                                                                   static_cast<float*>(V));
    timing_end(slot, s);
    CPC_LAUNCH_CHECK("subgrid_tc_kernel");
    return CPC_OK;
  }
  return launch_subgrid<float>(n, P->R_N, n_sub, S, sub, inv_h3, V, s);
}

extern "C" int lattice_interaction_energy(const cpc_kernel* P, const int* L, const int* edges, double Z, double* E_L,
                                          void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_MASTER)
    return fail(CPC_ERR_INVALID, "lattice_interaction_energy: needs a MASTER kernel");
  if (!L || !edges || !E_L) return fail(CPC_ERR_INVALID, "lattice_interaction_energy: NULL argument");
  if (!std::isfinite(Z)) return fail(CPC_ERR_INVALID, "lattice_interaction_energy: Z must be finite");
  const int n = P->n;
  Edges ed;
  int total = 0;
  for (int l = 0; l < 3; ++l) {
    if (L[l] < 0 || L[l] > kMaxLattice)
      return fail(CPC_ERR_UNSUPPORTED, "lattice_interaction_energy: L per axis must be in [0, 256]");
    ed.count[l] = L[l];
    for (int k = 0; k < L[l]; ++k) {
      const int e = edges[total + k];
      if (e < 1 || e > n - 1)
        return fail(CPC_ERR_INVALID, "lattice_interaction_energy: edge index outside [1, n-1]");
      ed.e[total + k] = e;
    }
    total += L[l];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // scratch: T [3][R_N] doubles and the list lengths, then the histograms
  // [3][2n] and the difference lists [3][2n][2]
  double* T = reinterpret_cast<double*>(P->d_lat);
  int* list_len = reinterpret_cast<int*>(P->d_lat + kEnergyListOff) - 4;
  int* ghist = reinterpret_cast<int*>(P->d_lat + kEnergyListOff);
  int* list = ghist + size_t(3) * 2 * n;
  const size_t hist_bytes = size_t(2) * n * sizeof(int);
  CPC_CUDA(cudaMemsetAsync(ghist, 0, 3 * hist_bytes, s));
  static std::atomic<int> pairs_smem{0};  // dynamic shared memory already allowed for lattice_pairs_kernel
  if (int(hist_bytes) > pairs_smem.load()) {
    CPC_CUDA(cudaFuncSetAttribute(lattice_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(hist_bytes)));
    pairs_smem.store(int(hist_bytes));
  }
  const int pslot = timing_begin("lattice_pairs_kernel", s);
  lattice_pairs_kernel<<<dim3(kPairChunks, 3), kPairThreads, hist_bytes, s>>>(n, ed, ghist);
  timing_end(pslot, s);
  CPC_LAUNCH_CHECK("lattice_pairs_kernel");
  lattice_diffs_kernel<<<3, kPairThreads, 0, s>>>(n, ghist, list, list_len);
  CPC_LAUNCH_CHECK("lattice_diffs_kernel");
  const int slot = timing_begin("lattice_energy_kernel", s);
  lattice_energy_kernel<<<dim3(P->R_N, 3), kEnergyThreads, 0, s>>>(n, P->R_N, P->d_p, list, list_len, T);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("lattice_energy_kernel");
  const double count = double(L[0]) * double(L[1]) * double(L[2]);
  const double scale = 0.5 * Z * Z / (P->h * P->h * P->h);
  lattice_energy_sum_kernel<<<1, 128, 0, s>>>(n, P->R_N, P->d_p, T, count, scale, E_L);
  CPC_LAUNCH_CHECK("lattice_energy_sum_kernel");
  return CPC_OK;
}
