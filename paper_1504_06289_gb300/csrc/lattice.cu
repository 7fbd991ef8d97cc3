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
//                     V[(s1,s2)][s3] is a product of a (pairs x q) matrix
//                     A = S1 * S2 and a (q x s3) matrix B = S3, each row split
//                     exactly into four bf16 integer slices under a per-row
//                     power of two (a published error-free splitting, the
//                     "Ozaki scheme"); the slice products are summed exactly
//                     in TMEM (every group sum over 64 q is an integer below
//                     2^24) and folded into float32 once per output.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cpc_internal.h"
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
constexpr int BM = 128;      // (s1, s2) pairs per CTA, one TMEM lane each
constexpr int BN = 64;       // s3 points per sub-tile
constexpr int NSL = 4;       // slices: x = 2^e (s0 2^-8 + s1 2^-16 + s2 2^-24 + s3 2^-32)
constexpr int THREADS = 128;
constexpr uint32_t A_SLICE = BM * 128, B_SLICE = BN * 128;  // rows of 64 bf16 (128 bytes)
constexpr uint32_t TMEM_COLS = 256;                         // NSL groups x BN columns
constexpr size_t kSmemBytes = size_t(NSL) * (A_SLICE + B_SLICE) + 1024 + 64;
constexpr long kSpinLimit = 20000000;

// row of 64 values (q = 0..63) -> NSL bf16 slices in 128-byte-swizzled K-major
// rows at `base` (slice k at base + k * slice_bytes); returns the row exponent
__device__ __forceinline__ int slice_row(const float (&x)[64], uint8_t* base, uint32_t slice_bytes, int row) {
  float m = 0.0f;
#pragma unroll
  for (int q = 0; q < 64; ++q) m = fmaxf(m, fabsf(x[q]));
  int e = 0;
  if (m > 0.0f) frexpf(m, &e);  // |x| < 2^e
#pragma unroll
  for (int c = 0; c < 8; ++c) {  // 16-byte chunk c holds q = 8c .. 8c+7
    uint32_t w[NSL][4];
#pragma unroll
    for (int h = 0; h < 8; h += 2) {
      float sl[NSL][2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float a = ldexpf(x[8 * c + h + u], 8 - e);  // |a| < 256
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
    const uint32_t off = umma::sw128_offset(row, c * 16);
#pragma unroll
    for (int k = 0; k < NSL; ++k)
      *reinterpret_cast<uint4*>(base + k * slice_bytes + off) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
  }
  return e;
}

constexpr int kMaxTiles = 512 / BN;                          // n_sub <= 512
constexpr size_t kBTileBytes = size_t(NSL) * B_SLICE;          // 32 KB per sub-tile
constexpr size_t kScratchBytes = kMaxTiles * kBTileBytes + 512 * sizeof(int);

// B rows (b_q = S3[q][i3], s3 = 0..n_sub-1) sliced once per call into the
// kernel's scratch: sub-tile j at j * 32 KB, slice k at + k * 8 KB, rows in the
// 128-byte-swizzled layout the MMA reads; exponents after the tiles.
__global__ void __launch_bounds__(BN)
slice_b_kernel(int n, int R_N, int n_sub, const double* __restrict__ S, const int* __restrict__ sub,
               unsigned char* __restrict__ scratch) {
  const int t = threadIdx.x, j = blockIdx.x, s3 = j * BN + t;
  const bool ok = s3 < n_sub;
  const int i3 = clamp_index(sub[2 * n_sub + (ok ? s3 : 0)], n);
  float x[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) x[q] = (ok && q < R_N) ? float(S[(size_t)(2 * R_N + q) * n + i3]) : 0.0f;
  const int e = slice_row(x, scratch + (size_t)j * kBTileBytes, B_SLICE, t);
  reinterpret_cast<int*>(scratch + kMaxTiles * kBTileBytes)[s3 < 512 ? s3 : 511] = ok ? e : 0;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__global__ void __launch_bounds__(THREADS)
subgrid_tc_kernel(int n, int R_N, int n_sub, const double* __restrict__ S, const int* __restrict__ sub,
                  float inv_h3, const unsigned char* __restrict__ scratch, float* __restrict__ V) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = umma::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t* smem = smem_raw + pad;
  const uint32_t sA = raw + pad, sB = sA + NSL * A_SLICE;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + NSL * (A_SLICE + B_SLICE));  // MMA done
  uint64_t* bbar = mbar + 1;                                                          // B tile landed
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(bbar + 1);
  const int* eB = reinterpret_cast<const int*>(scratch + kMaxTiles * kBTileBytes);

  const int t = threadIdx.x, warp = t >> 5;
  const long long n_pairs = (long long)n_sub * n_sub;
  const long long p = (long long)blockIdx.x * BM + t;  // this thread's pair and TMEM lane
  // A row: a_q = S1[q][i1] S2[q][i2] (float64 product, rounded once), q >= R_N zero
  int eA;
  {
    float x[64];
    const bool ok = p < n_pairs;
    const int s1 = ok ? int(p / n_sub) : 0, s2 = ok ? int(p % n_sub) : 0;
    const int i1 = clamp_index(sub[s1], n), i2 = clamp_index(sub[n_sub + s2], n);
#pragma unroll
    for (int q = 0; q < 64; ++q)
      x[q] = (ok && q < R_N) ? float(S[(size_t)q * n + i1] * S[(size_t)(R_N + q) * n + i2]) : 0.0f;
    eA = slice_row(x, smem, A_SLICE, t);
  }
  if (warp == 0) umma::tmem_alloc(tmem_ptr, TMEM_COLS);
  if (t == 0) {
    umma::mbar_init(mbar, 1);
    umma::mbar_init(bbar, 1);
    umma::mbar_fence_init();
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tbase = *tmem_ptr;
  const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * warp) << 16);
  constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN);
  bool ok_wait = true;
  const int n_tiles = (n_sub + BN - 1) / BN;
  umma::fence_proxy_async();  // the A slices (generic-proxy writes) -> tensor-core reads
  __syncthreads();
  for (int j = 0; j < n_tiles; ++j) {
    // the sub-tile's B slices (sliced once per call by slice_b_kernel): one bulk copy
    if (t == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(umma::smem_u32(bbar)),
                   "r"(uint32_t(kBTileBytes))
                   : "memory");
      bulk_load(sB, scratch + (size_t)j * kBTileBytes, uint32_t(kBTileBytes), umma::smem_u32(bbar));
    }
    ok_wait = ok_wait && umma::mbar_wait(bbar, j & 1, kSpinLimit);
    if (t == 0) {
      // group g accumulates the slice pairs (a, b) with a + b = g
#pragma unroll
      for (int g = 0; g < NSL; ++g) {
        uint32_t acc = 0;
#pragma unroll
        for (int a = 0; a <= g; ++a) {
          const int b = g - a;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            umma::mma_bf16(tbase + g * BN, umma::desc_k_sw128(sA + a * A_SLICE + kk * 32),
                           umma::desc_k_sw128(sB + b * B_SLICE + kk * 32), idesc, acc);
            acc = 1;
          }
        }
      }
      umma::mma_commit(mbar);
    }
    ok_wait = ok_wait && umma::mbar_wait(mbar, j & 1, kSpinLimit);
    umma::fence_after();
    // fold: v = (S0 + S1 2^-8 + S2 2^-16 + S3 2^-24) 2^(eA + eB - 16) h^-3
#pragma unroll
    for (int cb = 0; cb < BN / 16; ++cb) {
      float v0[16], v1[16], v2[16], v3[16];
      umma::tmem_ld16(lane_base + cb * 16, v0);
      umma::tmem_ld16(lane_base + BN + cb * 16, v1);
      umma::tmem_ld16(lane_base + 2 * BN + cb * 16, v2);
      umma::tmem_ld16(lane_base + 3 * BN + cb * 16, v3);
      umma::tmem_ld_wait();
      const int c0 = j * BN + cb * 16;
      if (p < n_pairs && c0 < n_sub) {
        float val[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float f = fmaf(v3[u], 1.0f / 16777216.0f,
                               fmaf(v2[u], 1.0f / 65536.0f, fmaf(v1[u], 1.0f / 256.0f, v0[u])));
          const int e = (c0 + u < n_sub) ? __ldg(eB + c0 + u) : 0;
          val[u] = ok_wait ? ldexpf(f, eA + e - 16) * inv_h3 : __int_as_float(0x7fc00000);
        }
        float* out = V + p * n_sub + c0;
        if ((n_sub & 15) == 0) {  // 16 values, 64-byte aligned: four 16-byte stores
#pragma unroll
          for (int u = 0; u < 16; u += 4)
            *reinterpret_cast<float4*>(out + u) = make_float4(val[u], val[u + 1], val[u + 2], val[u + 3]);
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (c0 + u < n_sub) out[u] = val[u];
        }
      }
    }
    umma::fence_before();
    __syncthreads();  // B slices and TMEM are rewritten by the next sub-tile
    umma::fence_after();
  }
  if (warp == 0) umma::tmem_dealloc(tbase, TMEM_COLS);
}
}  // namespace lat

size_t lattice_scratch_bytes() { return lat::kScratchBytes; }

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
    const long long blocks = ((long long)n_sub * n_sub + lat::BM - 1) / lat::BM;
    CPC_CUDA(cudaFuncSetAttribute(lat::subgrid_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(lat::kSmemBytes)));
    lat::slice_b_kernel<<<(n_sub + lat::BN - 1) / lat::BN, lat::BN, 0, s>>>(n, P->R_N, n_sub, S, sub, P->d_lat);
    CPC_LAUNCH_CHECK("slice_b_kernel");
    const int slot = timing_begin("subgrid_tc_kernel", s);
    lat::subgrid_tc_kernel<<<(unsigned)blocks, lat::THREADS, lat::kSmemBytes, s>>>(n, P->R_N, n_sub, S, sub,
                                                                                   float(inv_h3), P->d_lat,
                                                                                   static_cast<float*>(V));
    timing_end(slot, s);
    CPC_LAUNCH_CHECK("subgrid_tc_kernel");
    return CPC_OK;
  }
  return launch_subgrid<float>(n, P->R_N, n_sub, S, sub, inv_h3, V, s);
}
