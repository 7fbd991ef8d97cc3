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
// 256 cells S_0 and S_1 are integers of magnitude at most 2^24 (256 * 2^16
// each), so the bf16 MMAs accumulate them exactly in TMEM whatever the tensor
// core's rounding; S_2 (at most 256 * 81920 = 2.1e7) may pass 2^24, where a
// float32 accumulation step can round by 2^-24 of S_2, i.e. below 2^-38 of the
// 2^(e_r+e_s) scale of the entry.  Every 256 cells the accumulators are folded
// into a compensated float32 sum (TwoSum) per entry.
//
// Tiles: a CTA pair (2-CTA cluster, cta_group::2) computes 256 rows of U (M)
// x 128 rows of W (N) for one kernel term; each CTA streams its 128 U rows and
// 64 W rows with TMA (cp.async.bulk.tensor, 128-byte swizzle, completion
// counted on an mbarrier) through 3 shared-memory stages, and one thread of
// the even CTA issues the MMAs for both.  Sixteen warps per CTA read the
// accumulators after every four chunks; the three axes run as one stream of
// chunks and the running product over axes stays in TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "cpc_internal.h"
#include "umma.cuh"

namespace cpc {
namespace tc {

constexpr int BM = 128;      // U rows per CTA (M = 256 per CTA pair)
constexpr int BN = 128;      // W rows (output columns) per pair tile
constexpr int BNH = BN / 2;  // W rows loaded by each CTA of the pair
static_assert(BM == BN, "the symmetric E_H tiling uses square 128 x 128 blocks");
constexpr int BKC = 64;      // chunk of 64 cells = one 128-byte bf16 row
constexpr int READERS = 16;  // accumulator reader warps: lane quadrant x column quarter
constexpr int BNW = BN / 4;  // columns read by one reader warp
constexpr int THREADS = (READERS + 1) * 32;  // + one TMA/MMA warp
constexpr int STAGES = 3;
constexpr int GROUP = 4;  // 64-cell chunks per TMEM accumulation: S_0, S_1 over 256 cells stay within 2^24
constexpr uint32_t A_SLICE_BYTES = BM * 128, B_SLICE_BYTES = BNH * 128;
constexpr uint32_t STAGE_BYTES = 3 * A_SLICE_BYTES + 3 * B_SLICE_BYTES;  // 72 KB per CTA
constexpr uint32_t TMEM_COLS = 512;  // 3 groups x 128 columns, then the product over axes
constexpr uint32_t PROD_COL = 3 * BN;
// stages, alignment slack, barriers, then per-column exponents (3 axes) and coefficients
constexpr size_t kColBytes = 3 * BN * sizeof(int) + BN * sizeof(double);
constexpr size_t kRowBytes = 4 * BM * sizeof(double);  // rows mode: the 4 column quarters of each row
constexpr size_t kSmemBytes = size_t(STAGES) * STAGE_BYTES + 1024 + 256 + kColBytes + kRowBytes;
constexpr long kSpinLimit = 20000000;

// x -> (s0, s1, s2) with one exponent per row (2^e > max |x| over the row):
// one CTA of 256 threads per row, the row read once into registers
// (n / 256 values per thread, rounded up).
//
// Source rows are (l, s, q) of a [3][R_f][R_N][n] array (R_N = 1 for U).
// Slices are written chunk-blocked, so that the rows of one operand tile
// (64 consecutive s, one 64-cell chunk) are one contiguous block:
//   out[k][G = l*R_N + q][t][s][i % 64],  t = i / 64,  k = slice.
template <typename TS, int VPT>
__global__ void __launch_bounds__(256) slice_rows_kernel(const TS* __restrict__ src, long long rows, int n, int R_f,
                                                         int R_N, __nv_bfloat16* __restrict__ out,
                                                         long long slice_stride, int* __restrict__ expo) {
  __shared__ float red[8];
  const int T = n >> 6;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const TS* x = src + row * n;
    const long long per_l = (long long)R_f * R_N;
    const int l = (int)(row / per_l);
    const int rem = (int)(row - l * per_l);
    const int srow = rem / R_N, q = rem - srow * R_N;
    __nv_bfloat16* ob = out + ((long long)(l * R_N + q) * T * R_f + srow) * 64;
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
      __nv_bfloat16* o = ob + (long long)(i >> 6) * R_f * 64 + (i & 63);
      o[0] = __float2bfloat16_rn(s0);
      o[slice_stride] = __float2bfloat16_rn(s1);
      o[2 * slice_stride] = __float2bfloat16_rn(s2);
    }
    __syncthreads();  // red[] reused by the next row
  }
}

// E_H tiling of the symmetric Gram.  With nb = ceil(R_f / 128) blocks per
// side, the blocks {i, c}, i <= c, of 128 rows x 128 columns are what E_H
// needs; a CTA pair computes two blocks that share a column block.  Column c
// starts with its diagonal block and the blocks of rows i < c; walking
// c = nb-1 .. 1, a column with an odd count hands its block {c-1, c} to column
// c-1, where it is computed as rows c, columns c-1 (the transpose, equal by
// symmetry).  Every column but column 0 then holds an even count, so at most
// one CTA pair has a single block (about nb^2 / 4 pairs instead of the
// nb/2 x nb of a 256 x 128 tiling of the upper triangle).
__host__ __device__ inline int eh_pair_tiles(int nb) {
  int carry = 0, total = 0;
  for (int c = nb - 1; c >= 0; --c) {
    const int cnt = c + 1 + carry;
    const int out = (c > 0 && (cnt & 1)) ? 1 : 0;
    total += (cnt - out + 1) / 2;
    carry = out;
  }
  return total;
}
// row blocks (rb0, rb1; rb1 = -1: none) and column block of pair tile pt
__host__ __device__ inline void eh_pair_tile(int nb, int pt, int* rb0, int* rb1, int* cb) {
  int carry = 0, base = 0;
  for (int c = nb - 1; c >= 0; --c) {
    const int cnt = c + 1 + carry;
    const int out = (c > 0 && (cnt & 1)) ? 1 : 0;
    const int np = (cnt - out + 1) / 2;
    if (pt < base + np) {
      // rows of column c: 0..c without c-1 when handed on, then c+1 when received
      const int len_main = out ? c : c + 1;
      auto elem = [&](int e) {
        if (e < len_main) return (out && e >= c - 1) ? e + 1 : e;
        return (carry && e == len_main) ? c + 1 : -1;
      };
      const int e = 2 * (pt - base);
      *rb0 = elem(e);
      *rb1 = elem(e + 1);
      *cb = c;
      return;
    }
    base += np;
    carry = out;
  }
  *rb0 = -1;
  *rb1 = -1;
  *cb = 0;
}

struct Args {
  const int* eA;           // [3 * M] row exponents of the A rows (U or item factors), row l*M + r
  const int* eB;           // [3 * Ns * R_N] row exponents of W, row (l*Ns + s)*R_N + q
  int M, Ns, R_N, n;       // A rows, W factor columns, kernel terms, cells
  int rows_mode;           // 0: E_H (M == Ns, symmetric, upper triangle); 1: per-row sums
  const double* c;         // E_H: coefficients of rows and columns
  const double* c_col;     // column coefficients c_s
  double* partial;         // E_H: one sum per CTA; rows mode: [(q * n_ct + ct) * M + r]
  double* G;               // E_H only (may be NULL)
  int* status;
};

// 5D tiled TMA load into this CTA's shared memory; the innermost coordinate is
// always 0 (16-byte aligned); the mbarrier may be the peer CTA's (cta_group::2)
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c1, int c2, int c3,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, %3, %4, %5, %6}], [%7];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(c1), "r"(c2), "r"(c3), "r"(0), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// chunk tt of the stream (axis tt / T, cells (tt % T) * 64 ..) into stage tt % STAGES
// of this CTA; completion is counted on the even CTA's barrier (cluster address)
__device__ __forceinline__ void issue_stage(const CUtensorMap* mapA, const CUtensorMap* mapB, const Args& g,
                                            uint32_t sbase, uint32_t fullbar_cluster, int tt, int T, int q, int r0,
                                            int sb0) {
  const int l = tt / T, t = tt % T;
  const uint32_t stage = sbase + (tt % STAGES) * STAGE_BYTES;
  // all three slices of each operand tile in one copy: A dims (cell, r, t, l, slice),
  // B dims (cell, s, t, l*R_N + q, slice); rows past R_f read as zeros
  tma_load_5d(stage, mapA, r0, t, l, fullbar_cluster);
  tma_load_5d(stage + 3 * A_SLICE_BYTES, mapB, sb0, t, l * g.R_N + q, fullbar_cluster);
}

// the 6 slice-pair products of one chunk for the CTA pair (M = 256, N = 128)
__device__ __forceinline__ void issue_mmas(uint32_t stage, uint32_t tacc, uint32_t accumulate) {
  constexpr uint32_t idesc = umma::idesc_bf16_f32(2 * BM, BN);
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
        umma::mma_bf16_pair(tacc + g * BN, ad, bd, idesc, acc);
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

// One CTA pair (a 2-CTA cluster) per tile of 256 U rows x 128 W rows of one
// kernel term q.  Both CTAs stream their half of the operands (128 U rows, 64
// W rows) with TMA into their own shared memory and count the bytes on the
// even CTA's full barrier; one thread of the even CTA issues the pair MMAs
// (each CTA's TMEM receives its 128 rows x 128 columns).  In each CTA, warps
// 0-15 read the accumulators (warp w: TMEM lanes 32 (w % 4).., columns
// 32 (w / 4)..), warp 16 drives the copies.  Up to GROUP = 4 consecutive
// 64-cell chunks accumulate before each readout (S_0 and S_1 stay integers of
// magnitude at most 2^24 over 256 cells, so they are exact).
// Barriers: full[stage] (even CTA: both halves landed), sfree[stage] (both
// CTAs: the MMAs reading a stage finished), done (both CTAs: a group of
// chunks accumulated), freeb (even CTA: the 32 reader warps of the pair
// took the accumulators out of TMEM).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
gemm3_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Args g) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = umma::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t* smem = smem_raw + pad;
  const uint32_t sbase = raw + pad;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);  // [STAGES]
  uint64_t* sfree = full + STAGES;                                             // [STAGES]
  uint64_t* done = sfree + STAGES;                                             // [1]
  uint64_t* freeb = done + 1;                                                  // [1]
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(freeb + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_ptr + 1);
  double* col_c = reinterpret_cast<double*>(smem + STAGES * STAGE_BYTES + 256);  // [BN]
  int* col_e = reinterpret_cast<int*>(col_c + BN);                              // [3][BN]
  double* row_q = reinterpret_cast<double*>(col_e + 3 * BN);                    // [4][BM]
  __shared__ double red[THREADS / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = umma::cluster_ctarank();
  const int q = blockIdx.y;
  const int n_ct = (g.Ns + BN - 1) / BN;
  const int pair = blockIdx.x >> 1;
  int ct, r0;
  if (g.rows_mode) {  // rectangular: 256-row x 128-column pair tiles
    const int rp = pair / n_ct;
    ct = pair % n_ct;
    r0 = rp * 2 * BM + int(rank) * BM;
  } else {  // symmetric: two 128 x 128 blocks of one column block (above)
    int rb0, rb1;
    eh_pair_tile(n_ct, pair, &rb0, &rb1, &ct);
    const int rb = rank ? rb1 : rb0;
    r0 = (rb >= 0 ? rb : n_ct) * BM;  // no block: rows past R_f (read as zeros, never counted)
  }
  const int s0 = ct * BN, sb0 = s0 + int(rank) * BNH;
  const bool diag = !g.rows_mode && r0 == s0;  // a diagonal block: only r <= s counts
  // the tile's column coefficients and row exponents of W, once
  for (int i = tid; i < 4 * BN; i += THREADS) {
    const int j = i % BN, s = s0 + j;
    if (i < BN) col_c[j] = (s < g.Ns) ? g.c_col[s] : 0.0;
    else col_e[i - BN] = (s < g.Ns) ? g.eB[((long long)(i / BN - 1) * g.Ns + s) * g.R_N + q] : 0;
  }
  if (warp == 0) umma::tmem_alloc_pair(tmem_ptr, TMEM_COLS);
  if (tid == 32) {
    for (int i = 0; i < STAGES; ++i) {
      umma::mbar_init(&full[i], 1);
      umma::mbar_init(&sfree[i], 1);
    }
    umma::mbar_init(done, 1);
    umma::mbar_init(freeb, 2 * READERS);
    *abort_flag = 0;
    umma::mbar_fence_init();
  }
  umma::fence_before();
  __syncthreads();
  umma::cluster_sync();  // the peer's barriers are initialised before any copy or arrive reaches them
  umma::fence_after();
  const uint32_t tbase = *tmem_ptr;
  const int T = g.n / BKC, TT = 3 * T;  // chunks (T even)
  // chunks accumulate in TMEM in groups of up to GROUP (the last group of an
  // axis may be shorter); GA groups per axis, 3 GA in all
  const int GA = (T + GROUP - 1) / GROUP;
  const uint32_t freeb_even = umma::mapa(umma::smem_u32(freeb), 0);
  double sum = 0.0;

  if (warp == READERS) {
    if (lane == 0) {
      auto fullc = [&](int tt) { return umma::mapa(umma::smem_u32(&full[tt % STAGES]), 0); };
      if (rank == 0) {
        for (int tt = 0; tt < STAGES - 1 && tt < TT; ++tt) {
          mbar_expect_tx(umma::smem_u32(&full[tt]), 2 * STAGE_BYTES);
          issue_stage(&mapA, &mapB, g, sbase, fullc(tt), tt, T, q, r0, sb0);
        }
        for (int tt = 0; tt < TT; ++tt) {
          const int t = tt % T, gi = (tt / T) * GA + t / GROUP;  // group of this chunk
          const bool first = (t % GROUP == 0), last = (t % GROUP == GROUP - 1) || (t == T - 1);
          if (!wait_or_abort(&full[tt % STAGES], (tt / STAGES) & 1, abort_flag)) break;
          if (first && gi >= 1 && !wait_or_abort(freeb, (gi - 1) & 1, abort_flag)) break;
          umma::fence_after();
          issue_mmas(sbase + (tt % STAGES) * STAGE_BYTES, tbase, first ? 0u : 1u);
          umma::mma_commit_pair(&sfree[tt % STAGES]);
          if (last) umma::mma_commit_pair(done);
          const int tn = tt + STAGES - 1;
          if (tn < TT) {
            // stage tn % STAGES last held chunk tt - 1: wait until its MMAs finished
            if (tt >= 1 && !wait_or_abort(&sfree[(tt - 1) % STAGES], ((tt - 1) / STAGES) & 1, abort_flag)) break;
            mbar_expect_tx(umma::smem_u32(&full[tn % STAGES]), 2 * STAGE_BYTES);
            issue_stage(&mapA, &mapB, g, sbase, fullc(tn), tn, T, q, r0, sb0);
          }
        }
      } else {
        for (int tt = 0; tt < STAGES - 1 && tt < TT; ++tt) issue_stage(&mapA, &mapB, g, sbase, fullc(tt), tt, T, q, r0, sb0);
        for (int tt = 0; tt + STAGES - 1 < TT; ++tt) {
          const int tn = tt + STAGES - 1;
          if (tt >= 1 && !wait_or_abort(&sfree[(tt - 1) % STAGES], ((tt - 1) / STAGES) & 1, abort_flag)) break;
          issue_stage(&mapA, &mapB, g, sbase, fullc(tn), tn, T, q, r0, sb0);
        }
      }
      // drain: every commit of the pair has arrived on this CTA's stage barriers
      // before the CTA can leave
      if (!*abort_flag)
        for (int tt = (TT > STAGES ? TT - STAGES : 0); tt < TT; ++tt)
          if (!wait_or_abort(&sfree[tt % STAGES], (tt / STAGES) & 1, abort_flag)) break;
    }
  } else {
    const int quad = warp & 3, part = warp >> 2;
    const int r = r0 + 32 * quad + lane;  // this thread's row and TMEM lane
    const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * quad) << 16) + part * BNW;
    const int sh0 = s0 + part * BNW;  // first column of this warp
    // running sum of an axis as an unevaluated pair tot + lo (TwoSum per fold);
    // |lo| stays near 2^-24 |tot|, so lo is kept in bf16 (two per register):
    // its own rounding is then below 2^-32 |tot|
    float tot[BNW];
    __nv_bfloat162 lo[BNW / 2];
#pragma unroll
    for (int j = 0; j < BNW; ++j) tot[j] = 0.0f;
#pragma unroll
    for (int j = 0; j < BNW / 2; ++j) lo[j] = __float2bfloat162_rn(0.0f);
    double row = 0.0;
    bool ok = true;
    for (int gi = 0; gi < 3 * GA && ok; ++gi) {
      if (!wait_or_abort(done, gi & 1, abort_flag)) { ok = false; break; }
      umma::fence_after();
#pragma unroll
      for (int cb = 0; cb < BNW / 8; ++cb) {
        float v0[8], v1[8], v2[8];
        const uint32_t col = cb * 8;
        umma::tmem_ld8(lane_base + col, v0);
        umma::tmem_ld8(lane_base + col + BN, v1);
        umma::tmem_ld8(lane_base + col + 2 * BN, v2);
        umma::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          float e[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float v = fmaf(v2[j + h], 1.0f / 65536.0f, fmaf(v1[j + h], 1.0f / 256.0f, v0[j + h]));
            float& t = tot[cb * 8 + j + h];
            const float sm = t + v, bb = sm - t;
            e[h] = (t - (sm - bb)) + (v - bb);
            t = sm;
          }
          __nv_bfloat162& L = lo[(cb * 8 + j) / 2];
          const float2 f = __bfloat1622float2(L);
          L = __floats2bfloat162_rn(f.x + e[0], f.y + e[1]);
        }
      }
      umma::fence_before();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive_cluster(freeb_even);
      if (gi % GA == GA - 1) {
        // axis l finished: G_l = 2^(e_r + e_s - 16) (tot + lo); the running
        // product over axes lives in TMEM columns PROD_COL.. between axes
        const int l = gi / GA;
        const int er = (r < g.M) ? g.eA[l * g.M + r] : 0;
#pragma unroll
        for (int cb = 0; cb < BNW / 16; ++cb) {
          float pv[16];
          if (l > 0) {
            umma::tmem_ld16(lane_base + PROD_COL + cb * 16, pv);
            umma::tmem_ld_wait();
          }
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int j = cb * 16 + jj, s = sh0 + j;
            const int es = col_e[l * BN + part * BNW + j];
            const __nv_bfloat162 L = lo[j / 2];
            const float lj = (j & 1) ? __high2float(L) : __low2float(L);
            const float Gv = ldexpf(tot[j] + lj, er + es - 16);
            tot[j] = 0.0f;
            if (j & 1) lo[j / 2] = __float2bfloat162_rn(0.0f);
            const bool in = r < g.M && s < g.Ns && (!diag || r <= s);
            if (g.G && in) {
              double* Gq = g.G + ((size_t)l * gridDim.y + q) * (size_t)g.M * g.M;
              Gq[(size_t)r * g.M + s] = Gv;
              Gq[(size_t)s * g.M + r] = Gv;
            }
            const float pr = (l > 0) ? pv[jj] * Gv : Gv;
            pv[jj] = pr;
            if (l == 2 && in) {
              const double wgt = (g.rows_mode || r == s) ? 1.0 : 2.0;  // E_H: off-diagonal pairs twice
              row += wgt * col_c[part * BNW + j] * double(pr);
            }
          }
          if (l < 2) {
            umma::tmem_st16(lane_base + PROD_COL + cb * 16, pv);
            umma::tmem_st_wait();
          }
        }
      }
    }
    if (g.rows_mode) row_q[part * BM + 32 * quad + lane] = ok ? row : 0.0;
    else if (ok && r < g.M) sum = g.c[r] * row;
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) red[warp] = sum;
  umma::fence_before();
  __syncthreads();
  if (g.rows_mode) {
    // row sums of this CTA's 128 rows over the tile's 128 columns
    if (tid < BM && r0 + tid < g.M)
      g.partial[((size_t)q * n_ct + ct) * g.M + r0 + tid] =
          row_q[tid] + row_q[BM + tid] + row_q[2 * BM + tid] + row_q[3 * BM + tid];
    if (tid == 0 && *abort_flag) atomicExch(g.status, 1);
  } else if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    g.partial[(size_t)q * gridDim.x + blockIdx.x] = s;
    if (*abort_flag) atomicExch(g.status, 1);
  }
  umma::cluster_sync();  // neither CTA leaves (or frees TMEM) while the pair still works
  if (warp == 0) {
    umma::fence_after();
    umma::tmem_dealloc_pair(tbase, TMEM_COLS);
  }
}

template <typename TS>
int launch_slice(const TS* src, long long rows, int n, int R_f, int R_N, __nv_bfloat16* out, long long slice_stride,
                 int* expo, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<long long>(rows, 1 << 20);
  const int slot = timing_begin("slice_rows_kernel", s);
  switch ((n + 255) / 256) {
    case 1: slice_rows_kernel<TS, 1><<<grid, 256, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo); break;
    case 2: slice_rows_kernel<TS, 2><<<grid, 256, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo); break;
    case 4: slice_rows_kernel<TS, 4><<<grid, 256, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo); break;
    case 8: slice_rows_kernel<TS, 8><<<grid, 256, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo); break;
    case 16: slice_rows_kernel<TS, 16><<<grid, 256, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo); break;
    case 32: slice_rows_kernel<TS, 32><<<grid, 256, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo); break;
    default:
      timing_end(slot, s);
      return fail(CPC_ERR_UNSUPPORTED, "tensor-core contraction: n must be a power of two up to 8192");
  }
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("slice_rows_kernel");
  return CPC_OK;
}

}  // namespace tc

// one partial per CTA: 2 CTAs per pair tile of the symmetric tiling and kernel term
size_t tc_partials(int R_f, int R_N) {
  return size_t(2) * tc::eh_pair_tiles((R_f + tc::BN - 1) / tc::BN) * R_N;
}

// n a multiple of 128 (the convolution that writes the W slices needs n >= 128)
bool tc_supported(const cpc_kernel* P) { return P->n >= 2 * tc::BKC && P->n % (2 * tc::BKC) == 0; }

namespace {
// workspace of the tensor-core contraction of M A rows against Ns R_N W rows:
// A slices, W slices, row exponents of A and W, status word (each 256-aligned)
struct TcLayout {
  size_t a, b;  // slice elements of A and W (all 3 slices, 3 axes)
  size_t off_b, off_ea, off_eb, off_status, total;
};
TcLayout tc_layout(const cpc_kernel* P, int M, int Ns) {
  TcLayout L;
  L.a = size_t(3) * 3 * M * P->n;
  L.b = size_t(3) * 3 * size_t(Ns) * P->R_N * P->n;
  L.off_b = align256(2 * L.a);
  L.off_ea = L.off_b + align256(2 * L.b);
  L.off_eb = L.off_ea + align256(4 * size_t(3) * M);
  L.off_status = L.off_eb + align256(4 * size_t(3) * Ns * P->R_N);
  L.total = L.off_status + 256;
  return L;
}
}  // namespace

size_t tc_workspace(const cpc_kernel* P, int R_f) { return tc_layout(P, R_f, R_f).total; }
size_t tc_rows_workspace(const cpc_kernel* P, int M, int Ns) { return tc_layout(P, M, Ns).total; }
size_t tc_rows_groups(const cpc_kernel* P, int Ns) { return size_t((Ns + tc::BN - 1) / tc::BN) * P->R_N; }

// status (int) of the tc workspace
int* tc_status_ptr(const cpc_kernel* P, int R_f, void* ws) {
  return reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + tc_layout(P, R_f, R_f).off_status);
}
int* tc_rows_status_ptr(const cpc_kernel* P, int M, int Ns, void* ws) {
  return reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + tc_layout(P, M, Ns).off_status);
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

void tc_w_slices(const cpc_kernel* P, int R_f, void* ws, __nv_bfloat16** slices, long long* slice_stride,
                 int** expo) {
  const TcLayout L = tc_layout(P, R_f, R_f);
  unsigned char* w = static_cast<unsigned char*>(ws);
  *slices = reinterpret_cast<__nv_bfloat16*>(w + L.off_b);
  *slice_stride = (long long)(L.b / 3);
  *expo = reinterpret_cast<int*>(w + L.off_eb);
}

namespace {
// slices (unless W is already sliced), tensor maps and the launch
int launch_tc(const cpc_kernel* P, int M, int Ns, const double* U, const float* W, const double* c,
              const double* c_col, double* G, double* partial, void* ws, cudaStream_t s, bool w_sliced,
              int rows_mode) {
  const int n = P->n, R_N = P->R_N;
  const TcLayout L = tc_layout(P, M, Ns);
  unsigned char* w = static_cast<unsigned char*>(ws);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(w);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(w + L.off_b);
  int* eA = reinterpret_cast<int*>(w + L.off_ea);
  int* eB = reinterpret_cast<int*>(w + L.off_eb);
  int* status = reinterpret_cast<int*>(w + L.off_status);
  CPC_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
  int st0 = tc::launch_slice(U, 3LL * M, n, M, 1, As, (long long)(L.a / 3), eA, s);
  if (st0) return st0;
  if (!w_sliced) {  // else the convolution already wrote them (convolve_from_spectra_sliced)
    st0 = tc::launch_slice(W, 3LL * Ns * R_N, n, Ns, R_N, Bs, (long long)(L.b / 3), eB, s);
    if (st0) return st0;
  }

  EncodeTiledFn enc;
  int st = encode_fn(&enc);
  if (st) return st;
  CUtensorMap mapA, mapB;
  const int T = n / tc::BKC;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  {
    // [slice 3][l 3][t T][r M][64 cells]
    const cuuint64_t dims[5] = {64, (cuuint64_t)M, (cuuint64_t)T, 3, 3};
    const cuuint64_t row = 128, strides[4] = {row, row * M, row * M * T, row * M * T * 3};
    const cuuint32_t box[5] = {tc::BKC, tc::BM, 1, 1, 3};
    if (enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, As, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CPC_ERR_CUDA, "tensor map for the U slices");
  }
  {
    // [slice 3][l*R_N + q][t T][s Ns][64 cells]
    const cuuint64_t dims[5] = {64, (cuuint64_t)Ns, (cuuint64_t)T, (cuuint64_t)3 * R_N, 3};
    const cuuint64_t row = 128, strides[4] = {row, row * Ns, row * Ns * T, row * Ns * T * 3 * R_N};
    const cuuint32_t box[5] = {tc::BKC, tc::BNH, 1, 1, 3};
    if (enc(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, Bs, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CPC_ERR_CUDA, "tensor map for the V_H factor slices");
  }
  const int n_rp = (M + 2 * tc::BM - 1) / (2 * tc::BM), n_ct = (Ns + tc::BN - 1) / tc::BN;
  const long long gx = rows_mode ? 2LL * n_rp * n_ct : 2LL * tc::eh_pair_tiles(n_ct);
  if (gx > 0x7fffffffLL || R_N > 65535) return fail(CPC_ERR_UNSUPPORTED, "tensor-core contraction: grid too large");
  dim3 grid((unsigned)gx, R_N);  // clusters of 2 along x
  tc::Args args{eA, eB, M, Ns, R_N, n, rows_mode, c, c_col, partial, G, status};
  CPC_CUDA(cudaFuncSetAttribute(tc::gemm3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc::kSmemBytes)));
  const int slot = timing_begin("gemm3_tc_kernel", s);
  tc::gemm3_tc_kernel<<<grid, tc::THREADS, tc::kSmemBytes, s>>>(mapA, mapB, args);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("gemm3_tc_kernel");
  return CPC_OK;
}
}  // namespace

int launch_eh_tc(const cpc_kernel* P, int R_f, const double* U, const float* W, const double* c, double* G,
                 double* partial, void* ws, cudaStream_t s, bool w_sliced) {
  return launch_tc(P, R_f, R_f, U, W, c, c, G, partial, ws, s, w_sliced, 0);
}

// Coulomb-matrix rows: rowpart[(q * n_ct + ct) * M + r] = sum over the 128
// columns s of tile ct of c_s prod_l G_l[r][s, q] (M item factors, Ns = R_rho)
int launch_rows_tc(const cpc_kernel* P, int M, const double* U_items, int Ns, const float* W_rho,
                   const double* c_rho, double* rowpart, void* ws, cudaStream_t s) {
  return launch_tc(P, M, Ns, U_items, W_rho, nullptr, c_rho, nullptr, rowpart, ws, s, false, 1);
}

}  // namespace cpc
