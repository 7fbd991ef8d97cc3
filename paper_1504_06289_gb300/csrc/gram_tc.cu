// float32-form E_H contraction on the tensor cores (tcgen05, kind::f16).
//
// Same quantity as gemm3a_kernel (Sec. 3.2 Eq. Factor_Mk_Conv, Sec. 2.5
// Eq. scal): G_l[r][s] = sum_i U_l[r][i] W_l[s*R_N+q][i], then
// sum_{r<=s} (1 or 2) c_r c_s prod_l G_l[r][s].
//
// Exact slicing.  Every operand row x (a column of U or of the V_H factors,
// as float32) is written as x = 2^e * (s0 2^-8 + s1 2^-16 + s2 2^-24) with
// 2^e > max|x| and integer slices |s0| <= 256, |s1|, |s2| <= 128, stored as
// bf16 (exact).  A product of two rows is
//   2^(e_r + e_s - 16) * (S0 + S1 2^-8 + S2 2^-16),  S_g = sum_{a+b=g} sum_i s_a s_b,
// dropping the a+b >= 3 terms (below float32 rounding of the operands).  Over
// 128 cells every S_g is an integer below 2^24, so the bf16 MMAs accumulate
// exactly in TMEM whatever the tensor core's rounding; every 128 cells the
// accumulators are folded into float32 registers (round to nearest).
//
// Tiles: 128 rows of U (M) x 64 columns of W (N), 128 threads (one TMEM lane
// per row).  One thread streams the operand slices with TMA
// (cp.async.bulk.tensor, 128-byte swizzle, completion counted on an
// mbarrier) through 3 shared-memory stages and issues the MMAs; two TMEM
// accumulator sets alternate so the readout of chunk t-1 by all threads
// overlaps the MMAs of chunk t.  The three axes run as one stream of chunks.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "cpc_internal.h"
#include "umma.cuh"

namespace cpc {
namespace tc {

constexpr int BM = 128, BN = 64, BKC = 64;  // chunk of 64 cells = one 128-byte bf16 row
constexpr int THREADS = 160, STAGES = 3;  // 4 reader warps + 1 TMA/MMA warp
constexpr uint32_t A_SLICE_BYTES = BM * 128, B_SLICE_BYTES = BN * 128;
constexpr uint32_t STAGE_BYTES = 3 * A_SLICE_BYTES + 3 * B_SLICE_BYTES;  // 73728
constexpr uint32_t TMEM_COLS = 512;  // 2 sets x 3 groups x 64, then the product over axes
constexpr uint32_t PROD_COL = 2 * 3 * BN;
constexpr size_t kSmemBytes = size_t(STAGES) * STAGE_BYTES + 1024 + 256;
constexpr long kSpinLimit = 20000000;

// x -> (s0, s1, s2) with one exponent per row (2^e > max |x| over the row):
// one CTA of 256 threads per row, the row read once into registers
// (n / 256 values per thread, n a multiple of 1024 or handled by a tail).
template <typename TS, int VPT>
__global__ void __launch_bounds__(256) slice_rows_kernel(const TS* __restrict__ src, long long rows, int n,
                                                         __nv_bfloat16* __restrict__ out, long long slice_stride,
                                                         int* __restrict__ expo) {
  __shared__ float red[8];
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const TS* x = src + row * n;
    float v[VPT];
    float m = 0.0f;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int i = (k * 256 + threadIdx.x);  // coalesced
      v[k] = (i < n) ? float(x[i]) : 0.0f;
      m = fmaxf(m, fabsf(v[k]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    float mm = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mm = fmaxf(mm, red[w]);
    int e = 0;
    if (mm > 0.0f) frexpf(mm, &e);  // mm = f 2^e, f in [0.5, 1): |x| < 2^e
    if (threadIdx.x == 0) expo[row] = e;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int i = k * 256 + threadIdx.x;
      if (i >= n) continue;
      const float a = ldexpf(v[k], 8 - e);  // |a| < 256
      const float s0 = rintf(a);
      const float b = (a - s0) * 256.0f;    // exact
      const float s1 = rintf(b);
      const float s2 = rintf((b - s1) * 256.0f);
      __nv_bfloat16* o = out + row * n + i;
      o[0] = __float2bfloat16_rn(s0);
      o[slice_stride] = __float2bfloat16_rn(s1);
      o[2 * slice_stride] = __float2bfloat16_rn(s2);
    }
    __syncthreads();  // red[] reused by the next row
  }
}

struct Args {
  const int* eA;           // [3 * R_f] row exponents of U, row l*R_f + r
  const int* eB;           // [3 * R_f * R_N] row exponents of W, row (l*R_f + s)*R_N + q
  int R_f, R_N, n;
  const double* c;
  double* partial;
  double* G;
  int* status;
};

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// chunk tt of the stream (axis tt / T, cells (tt % T) * 64 ..) into stage tt % STAGES
__device__ __forceinline__ void issue_stage(const CUtensorMap* mapA, const CUtensorMap* mapB, const Args& g,
                                            uint32_t sbase, uint32_t fullbar, int tt, int T, int q, int r0, int s0) {
  const int l = tt / T, k0 = (tt % T) * BKC;
  const uint32_t stage = sbase + (tt % STAGES) * STAGE_BYTES;
  mbar_expect_tx(fullbar, STAGE_BYTES);
#pragma unroll
  for (int a = 0; a < 3; ++a)  // A rows: slice a, axis l, rows r0.. (dim 1 = a*3R_f + l*R_f + r)
    tma_load_2d(stage + a * A_SLICE_BYTES, mapA, k0, (a * 3 + l) * g.R_f + r0, fullbar);
#pragma unroll
  for (int b = 0; b < 3; ++b)  // B rows: slice b, axis l, columns s0.., term q (dims: cell, q, b*3R_f + l*R_f + s)
    tma_load_3d(stage + 3 * A_SLICE_BYTES + b * B_SLICE_BYTES, mapB, k0, q, (b * 3 + l) * g.R_f + s0, fullbar);
}

__device__ __forceinline__ void issue_mmas(uint32_t stage, uint32_t tacc, uint32_t accumulate) {
  constexpr uint32_t idesc = umma::idesc_bf16_f32(BM, BN);
  const uint32_t a0 = stage, b0 = stage + 3 * A_SLICE_BYTES;
  // group g accumulates the slice pairs (a, b) with a + b = g
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    uint32_t acc = accumulate;
#pragma unroll
    for (int a = 0; a <= g; ++a) {
      const int b = g - a;
#pragma unroll
      for (int kk = 0; kk < BKC / 16; ++kk) {
        const uint64_t ad = umma::desc_k_sw128(a0 + a * A_SLICE_BYTES + kk * 32);
        const uint64_t bd = umma::desc_k_sw128(b0 + b * B_SLICE_BYTES + kk * 32);
        umma::mma_bf16(tacc + g * BN, ad, bd, idesc, acc);
        acc = 1;
      }
    }
  }
}

__device__ __forceinline__ bool wait_or_abort(uint64_t* mbar, uint32_t parity, volatile int* abort_flag) {
  uint32_t done = 0;
  for (long it = 0; it < kSpinLimit; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(umma::smem_u32(mbar)), "r"(parity));
    if (done) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// Warps 0-3 read the accumulators (one TMEM lane per thread); warp 4 (lane 0)
// streams the operands with TMA and issues the MMAs.  Two consecutive 64-cell
// chunks accumulate into the same TMEM set (every group sum stays an integer
// below 2^24 over 128 cells, so it is exact), which halves the readouts.
// Barriers: full[stage] (TMA bytes landed), sfree[stage] (the MMAs reading
// a stage finished), done[set] (both chunks of a pair accumulated),
// free[set] (the four reader warps took the set out of TMEM).
__global__ void __launch_bounds__(THREADS, 1)
gemm3_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Args g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = umma::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t* smem = smem_raw + pad;
  const uint32_t sbase = raw + pad;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);  // [STAGES]
  uint64_t* sfree = full + STAGES;                                             // [STAGES]
  uint64_t* done = sfree + STAGES;                                             // [2]
  uint64_t* freeb = done + 2;                                                  // [2]
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(freeb + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_ptr + 1);
  __shared__ double red[THREADS / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = blockIdx.y;
  const int n_ct = (g.R_f + BN - 1) / BN;
  const int rt = blockIdx.x / n_ct, ct = blockIdx.x % n_ct;
  const int r0 = rt * BM, s0 = ct * BN;
  if (r0 > s0 + BN - 1) {  // entirely below the diagonal of the symmetric sum
    if (tid == 0) g.partial[(size_t)q * gridDim.x + blockIdx.x] = 0.0;
    return;
  }
  if (warp == 0) umma::tmem_alloc(tmem_ptr, TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) {
      umma::mbar_init(&full[i], 1);
      umma::mbar_init(&sfree[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&done[i], 1);
      umma::mbar_init(&freeb[i], 4);
    }
    *abort_flag = 0;
    umma::mbar_fence_init();
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tbase = *tmem_ptr;
  const int T = g.n / BKC, TT = 3 * T;  // chunks (T even)
  const int PP = TT / 2, PA = T / 2;    // pairs in all, per axis
  double sum = 0.0;

  if (warp == 4) {
    if (lane == 0) {
      for (int tt = 0; tt < STAGES - 1 && tt < TT; ++tt)
        issue_stage(&mapA, &mapB, g, sbase, umma::smem_u32(&full[tt % STAGES]), tt, T, q, r0, s0);
      for (int tt = 0; tt < TT; ++tt) {
        const int pp = tt >> 1, set = pp & 1;
        if (!wait_or_abort(&full[tt % STAGES], (tt / STAGES) & 1, abort_flag)) break;
        if ((tt & 1) == 0 && pp >= 2 && !wait_or_abort(&freeb[set], ((pp - 2) >> 1) & 1, abort_flag)) break;
        umma::fence_after();
        issue_mmas(sbase + (tt % STAGES) * STAGE_BYTES, tbase + set * 3 * BN, (tt & 1) ? 1u : 0u);
        umma::mma_commit(&sfree[tt % STAGES]);
        if (tt & 1) umma::mma_commit(&done[set]);
        const int tn = tt + STAGES - 1;
        if (tn < TT) {
          // stage tn % STAGES last held chunk tt - 1: wait until its MMAs finished
          if (tt >= 1 && !wait_or_abort(&sfree[(tt - 1) % STAGES], ((tt - 1) / STAGES) & 1, abort_flag)) break;
          issue_stage(&mapA, &mapB, g, sbase, umma::smem_u32(&full[tn % STAGES]), tn, T, q, r0, s0);
        }
      }
    }
  } else {
    const int r = r0 + tid;  // this thread's row and TMEM lane
    const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * warp) << 16);
    // running sum of an axis as an unevaluated pair tot + lo (TwoSum per fold)
    float tot[BN], lo[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) { tot[j] = 0.0f; lo[j] = 0.0f; }
    double row = 0.0;
    bool ok = true;
    for (int pp = 0; pp < PP && ok; ++pp) {
      const int set = pp & 1;
      if (!wait_or_abort(&done[set], (pp >> 1) & 1, abort_flag)) { ok = false; break; }
      umma::fence_after();
#pragma unroll
      for (int cb = 0; cb < BN / 16; ++cb) {
        float v0[16], v1[16], v2[16];
        const uint32_t col = set * 3 * BN + cb * 16;
        umma::tmem_ld16(lane_base + col, v0);
        umma::tmem_ld16(lane_base + col + BN, v1);
        umma::tmem_ld16(lane_base + col + 2 * BN, v2);
        umma::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float v = fmaf(v2[j], 1.0f / 65536.0f, fmaf(v1[j], 1.0f / 256.0f, v0[j]));
          float& t = tot[cb * 16 + j];
          const float sm = t + v, bb = sm - t;
          lo[cb * 16 + j] += (t - (sm - bb)) + (v - bb);
          t = sm;
        }
      }
      umma::fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(umma::smem_u32(&freeb[set])));
      if (pp % PA == PA - 1) {
        // axis l finished: G_l = 2^(e_r + e_s - 16) (tot + lo); the running
        // product over axes lives in TMEM columns PROD_COL.. between axes
        const int l = pp / PA;
        const int er = (r < g.R_f) ? g.eA[l * g.R_f + r] : 0;
#pragma unroll
        for (int cb = 0; cb < BN / 16; ++cb) {
          float pv[16];
          if (l > 0) {
            umma::tmem_ld16(lane_base + PROD_COL + cb * 16, pv);
            umma::tmem_ld_wait();
          }
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = cb * 16 + jj, s = s0 + j;
            const int es = (s < g.R_f) ? __ldg(g.eB + ((long long)l * g.R_f + s) * g.R_N + q) : 0;
            const float Gv = ldexpf(tot[j] + lo[j], er + es - 16);
            tot[j] = 0.0f;
            lo[j] = 0.0f;
            const bool in = r < g.R_f && s < g.R_f && r <= s;
            if (g.G && in) {
              double* Gq = g.G + ((size_t)l * gridDim.y + q) * (size_t)g.R_f * g.R_f;
              Gq[(size_t)r * g.R_f + s] = Gv;
              Gq[(size_t)s * g.R_f + r] = Gv;
            }
            const float pr = (l > 0) ? pv[jj] * Gv : Gv;
            pv[jj] = pr;
            if (l == 2 && in) row += (r == s ? 1.0 : 2.0) * g.c[s] * double(pr);
          }
          if (l < 2) {
            umma::tmem_st16(lane_base + PROD_COL + cb * 16, pv);
            umma::tmem_st_wait();
          }
        }
      }
    }
    if (ok && r < g.R_f) sum = g.c[r] * row;
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) red[warp] = sum;
  umma::fence_before();
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    g.partial[(size_t)q * gridDim.x + blockIdx.x] = s;
    if (*abort_flag) atomicExch(g.status, 1);
  }
  if (warp == 0) {
    umma::fence_after();
    umma::tmem_dealloc(tbase, TMEM_COLS);
  }
}

template <typename TS>
int launch_slice(const TS* src, long long rows, int n, __nv_bfloat16* out, long long slice_stride, int* expo,
                 cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<long long>(rows, 1 << 20);
  switch ((n + 255) / 256) {
    case 1: slice_rows_kernel<TS, 1><<<grid, 256, 0, s>>>(src, rows, n, out, slice_stride, expo); break;
    case 2: slice_rows_kernel<TS, 2><<<grid, 256, 0, s>>>(src, rows, n, out, slice_stride, expo); break;
    case 4: slice_rows_kernel<TS, 4><<<grid, 256, 0, s>>>(src, rows, n, out, slice_stride, expo); break;
    case 8: slice_rows_kernel<TS, 8><<<grid, 256, 0, s>>>(src, rows, n, out, slice_stride, expo); break;
    case 16: slice_rows_kernel<TS, 16><<<grid, 256, 0, s>>>(src, rows, n, out, slice_stride, expo); break;
    case 32: slice_rows_kernel<TS, 32><<<grid, 256, 0, s>>>(src, rows, n, out, slice_stride, expo); break;
    default: return fail(CPC_ERR_UNSUPPORTED, "tensor-core contraction: n must be a power of two up to 8192");
  }
  CPC_LAUNCH_CHECK("slice_rows_kernel");
  return CPC_OK;
}

}  // namespace tc

size_t tc_partials(int R_f, int R_N) {
  const int n_rt = (R_f + tc::BM - 1) / tc::BM, n_ct = (R_f + tc::BN - 1) / tc::BN;
  return size_t(n_rt) * n_ct * R_N;
}

// two 64-cell chunks per accumulation: n a multiple of 128
bool tc_supported(const cpc_kernel* P) { return P->n >= 2 * tc::BKC && P->n % (2 * tc::BKC) == 0; }

// bytes: A slices, B slices, row exponents of A and B, status word (each 256-aligned)
size_t tc_workspace(const cpc_kernel* P, int R_f) {
  const size_t a = size_t(3) * 3 * R_f * P->n, b = size_t(3) * 3 * R_f * P->R_N * P->n;
  return align256(2 * a) + align256(2 * b) + align256(4 * size_t(3) * R_f) + align256(4 * size_t(3) * R_f * P->R_N) +
         256;
}

// status (int) at the end of the tc workspace
int* tc_status_ptr(const cpc_kernel* P, int R_f, void* ws) {
  return reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + tc_workspace(P, R_f) - 256);
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int encode_fn(EncodeTiledFn* out) {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  static int status = CPC_OK;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) status = CPC_ERR_CUDA;
    fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  if (status) return fail(status, "cuTensorMapEncodeTiled entry point unavailable");
  *out = fn;
  return CPC_OK;
}

int launch_eh_tc(const cpc_kernel* P, int R_f, const double* U, const float* W, const double* c, double* G,
                 double* partial, void* ws, cudaStream_t s) {
  const int n = P->n, R_N = P->R_N;
  const size_t a = size_t(3) * 3 * R_f * n, b = size_t(3) * 3 * R_f * R_N * n;
  unsigned char* w = static_cast<unsigned char*>(ws);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(w);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(w + align256(2 * a));
  int* eA = reinterpret_cast<int*>(w + align256(2 * a) + align256(2 * b));
  int* eB = reinterpret_cast<int*>(w + align256(2 * a) + align256(2 * b) + align256(4 * size_t(3) * R_f));
  int* status = tc_status_ptr(P, R_f, ws);
  CPC_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
  const long long arows = 3LL * R_f, brows = 3LL * R_f * R_N;
  int st0 = tc::launch_slice(U, arows, n, As, a / 3, eA, s);
  if (st0) return st0;
  st0 = tc::launch_slice(W, brows, n, Bs, b / 3, eB, s);
  if (st0) return st0;

  EncodeTiledFn enc;
  int st = encode_fn(&enc);
  if (st) return st;
  CUtensorMap mapA, mapB;
  {
    const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)9 * R_f};
    const cuuint64_t strides[1] = {(cuuint64_t)n * 2};
    const cuuint32_t box[2] = {tc::BKC, tc::BM};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, As, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CPC_ERR_CUDA, "tensor map for the U slices");
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)R_N, (cuuint64_t)9 * R_f};
    const cuuint64_t strides[2] = {(cuuint64_t)n * 2, (cuuint64_t)R_N * n * 2};
    const cuuint32_t box[3] = {tc::BKC, 1, tc::BN};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Bs, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CPC_ERR_CUDA, "tensor map for the V_H factor slices");
  }
  const int n_rt = (R_f + tc::BM - 1) / tc::BM, n_ct = (R_f + tc::BN - 1) / tc::BN;
  dim3 grid(n_rt * n_ct, R_N);
  tc::Args args{eA, eB, R_f, R_N, n, c, partial, G, status};
  CPC_CUDA(cudaFuncSetAttribute(tc::gemm3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc::kSmemBytes)));
  tc::gemm3_tc_kernel<<<grid, tc::THREADS, tc::kSmemBytes, s>>>(mapA, mapB, args);
  CPC_LAUNCH_CHECK("gemm3_tc_kernel");
  return CPC_OK;
}

}  // namespace cpc
