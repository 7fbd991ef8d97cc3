// E_H contraction on the tensor cores (tcgen05, kind::f16): the float32 form
// and the float64-accurate form CPC_FP64_TC.
//
// Same quantity as gemm3a_kernel and tri_gram_kernel (Sec. 3.2 Eq.
// Factor_Mk_Conv, Sec. 2.5 Eq. scal): G_l[r][s] = sum_i U_l[r][i] W_l[s*R_N+q][i],
// then sum_{r<=s} (1 or 2) c_r c_s prod_l G_l[r][s].
//
// Exact slicing (error-free splitting of the operands into low-precision
// slices, Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 2012).  Every
// operand row x (a column of U or of the V_H factors) is written as
//   x = 2^(e-8) * sum_k t_k,  t_k = s_k 2^(-8k),
// with integer digits s_k, each t_k exact in bf16.  A product of two rows is
// 2^(e_r + e_s - 16) sum_{a,b} sum_i t_a t_b.
//   * float32 form (NS = 3 slices of the float32 operands): U rows with
//     2^e > max|x|, |s_0| <= 256, |s_1|, |s_2| <= 128 (24 bits, error <=
//     2^-24 max|x|); W rows with balanced digits, 2^e > 2 max|x| and
//     |s_k| <= 128 for every k (23 bits, error <= 2^-23 max|x|, below the
//     float32 FFT's own error).  The pairs a + b <= 2 (6 products per cell);
//     the dropped ones lie below float32 rounding of the operands.  Three
//     TMEM accumulators per output: S_0 = sum s_0 s_0' (<= 2^15 per cell) is
//     an integer of magnitude at most 2^24 over 512 cells, exact in the bf16
//     MMAs whatever the tensor core's rounding; S_1 = sum (s_0 s_1' + s_1 s_0')
//     (<= 1.5 x 2^15 per cell, its digits being rounding remainders of both
//     signs) stays below 2^24 unless nearly every cell carries maximal digits
//     of one sign, and otherwise rounds by at most one unit (weight 2^-8) per
//     step: 2^-26 of the entry scale after the 64 steps of 512 cells; S_2
//     (a + b = 2, weight 2^-16) rounds by at most two units per step, 2^-39 of
//     the entry scale.  The weights 2^-8, 2^-16 are applied at readout, every
//     512 cells, into a compensated float32 sum (TwoSum) per entry.
//   * CPC_FP64_TC (NS = 5 slices of the float64 operands): 2^e > max|x|,
//     |s_0| <= 256, |s_k| <= 128 (40 bits of the row maximum); the pairs
//     a + b <= 4 (15 products per cell), the dropped ones below 2^-40 of the
//     row scales.  The slices are stored weighted (t_k), so each product
//     carries its weight; four accumulators per output: S_0 and S_1 exact over
//     256 cells as above (<= 2^16 and 1.5 x 2^15 per cell), S_2 (a + b = 2,
//     at most 5 x 2^22 units of 2^-16: one unit of rounding per step, 2^-40 of
//     the entry scale) and S_3 (a + b = 3, 4; weight <= 2^-24); folded every
//     256 cells into an unevaluated float pair per entry (TwoSum, ~48 bits).
//
// Tiles: a CTA pair (2-CTA cluster, cta_group::2) computes 256 rows of U (M)
// x 128 rows of W (N) for one kernel term; each CTA streams its 128 U rows and
// 64 W rows with TMA (cp.async.bulk.tensor, 128-byte swizzle for 64-cell
// chunks, 64-byte swizzle for the 32-cell chunks of CPC_FP64_TC; completion
// counted on an mbarrier) through 3 shared-memory stages, and one thread of
// the even CTA issues the MMAs for both.  Sixteen warps per CTA read the
// accumulators after every 512 (float32 form) or 256 cells.  Float32 form: the three axes run as
// one stream of chunks and the running product over axes stays in TMEM.
// CPC_FP64_TC: the readers write the float64 convolution matrices G, and
// E_H is reduced from them by a separate kernel.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <type_traits>

#include "cpc_internal.h"
#include "slice64.cuh"
#include "umma.cuh"

namespace cpc {
namespace tc {

constexpr int BM = 128;      // U rows per CTA (M = 256 per CTA pair)
constexpr int BN = 128;      // W rows (output columns) per pair tile
constexpr int BNH = BN / 2;  // W rows loaded by each CTA of the pair
static_assert(BM == BN, "the symmetric E_H tiling uses square 128 x 128 blocks");
static_assert(BN == 128, "TMEM: 4 accumulators or 3 + the product over axes, 128 columns each");
constexpr int READERS = 16;  // accumulator reader warps: lane quadrant x column quarter
constexpr int BNW = BN / 4;  // columns read by one reader warp
constexpr int THREADS = (READERS + 2) * 32;  // + the MMA warp + the TMA warp
constexpr uint32_t TMEM_COLS = 512;  // 3 groups x 128 columns, then the product over axes
constexpr uint32_t PROD_COL = 3 * BN;
// per-column exponents (3 axes) and coefficients; rows mode: the 4 column quarters of each row
constexpr size_t kColBytes = 3 * BN * sizeof(int) + BN * sizeof(double);
constexpr size_t kRowBytes = 4 * BM * sizeof(double);
constexpr long kSpinLimit = 20000000;

// Shapes of one form: NS slices per operand, BKC cells per chunk (one
// swizzled shared-memory row of BKC bf16: 128 or 64 bytes).
template <int NS_, int BKC_, int NACC_, int STAGES_, bool BAL_>
struct Form {
  static constexpr int NS = NS_, BKC = BKC_;
  static constexpr int NACC = NACC_;        // TMEM accumulators of BN columns per output tile
  static constexpr int STAGES = STAGES_;    // shared-memory stages of one chunk each
  static constexpr bool BAL = BAL_;         // balanced digits of W (the B operand): 2^e > 2 max|x|, |s_0| <= 128
  // cells per TMEM accumulation (S_0 exact, S_1 within 2^24 but for extreme data)
  static constexpr int EXACT_CELLS = BAL ? 512 : 256;
  static constexpr uint32_t ROW = BKC * 2;  // bytes per operand row of a chunk
  static constexpr int K_STEPS = BKC / 16;  // MMAs of K = 16 per slice pair and chunk
  static constexpr uint32_t A_SLICE_BYTES = BM * ROW, B_SLICE_BYTES = BNH * ROW;
  static constexpr uint32_t STAGE_BYTES = NS * (A_SLICE_BYTES + B_SLICE_BYTES);
  static constexpr int GROUP = EXACT_CELLS / BKC;  // chunks per TMEM accumulation
  static constexpr size_t SMEM = size_t(STAGES_) * STAGE_BYTES + 1024 + 256 + kColBytes + kRowBytes;
  static_assert(SMEM <= 232448, "shared memory of one CTA");
  static_assert((2 * STAGES + 3) * 8 <= 256, "barriers fit before the column data");
};
// float32 form: 3 stages of 64-cell chunks (72 KB), S_0..S_2 + the product over
// axes, balanced digits of W (readout every 512 cells; 12% faster than every
// 256 cells at density600_n8192).  (6 stages of 32-cell
// chunks, 36 KB, measured 32% slower at density600_n8192 and 30% slower in
// the Coulomb rows mode.)
using Form32 = Form<3, 64, 3, 3, true>;
// CPC_FP64_TC: 3 stages of 32-cell chunks (60 KB), S_0..S_3 (no product over axes)
using Form64 = Form<5, 32, 4, 3, false>;

// K-major operand descriptor for 128- or 64-byte swizzled rows (8-row atoms)
template <uint32_t ROW>
__device__ __forceinline__ uint64_t desc_k(uint32_t saddr) {
  static_assert(ROW == 128 || ROW == 64, "swizzle width");
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>(1) << 16;
  d |= static_cast<uint64_t>((8 * ROW) >> 4) << 32;  // stride between 8-row atoms
  d |= static_cast<uint64_t>(1) << 46;
  d |= static_cast<uint64_t>(ROW == 128 ? 2 : 4) << 61;  // SWIZZLE_128B / SWIZZLE_64B
  return d;
}

// Float32 form: x -> 3 slices with one exponent per row: one CTA of 256
// threads per row (several CTAs per SM keep rows in flight across each CTA's
// row barrier; one 1024-thread CTA per SM measured 2x slower), the row read
// once into registers (n / 256 values per thread, rounded up), rounded to
// float32, then its digits s_k stored as integers; BAL:
// balanced digits (2^e > 2 max|x|, the W operand), else 2^e > max|x| (U).
//
// Source rows are (l, s, q) of a [3][R_f][R_N][n] array (R_N = 1 for U).
// Slices are written chunk-blocked, so that the rows of one operand tile
// (64 consecutive s, one BKC-cell chunk) are one contiguous block:
//   out[k][G = l*R_N + q][t][s][i % BKC],  t = i / BKC,  k = slice.
// With qmap, row number `row` is taken from source row
// (row / n_qmap) R_N_src + qmap[row % n_qmap]: a subset of the kernel terms
// of a [..][R_N_src][n] array, compacted.
template <typename TS, int VPT, class F, int TPB, bool BAL>
__global__ void __launch_bounds__(TPB) slice_rows_kernel(const TS* __restrict__ src, long long rows, int n, int R_f,
                                                         int R_N, __nv_bfloat16* __restrict__ out,
                                                         long long slice_stride, int* __restrict__ expo,
                                                         const int* __restrict__ qmap, int n_qmap, int R_N_src) {
  constexpr int NS = F::NS, BKC = F::BKC;
  static_assert(NS == 3, "float32 form: three slices");
  __shared__ float red[TPB / 32];
  const int T = n / BKC;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const long long srow_src = qmap ? (row / n_qmap) * R_N_src + __ldg(qmap + row % n_qmap) : row;
    const TS* x = src + srow_src * n;
    const long long per_l = (long long)R_f * R_N;
    const int l = (int)(row / per_l);
    const int rem = (int)(row - l * per_l);
    const int srow = rem / R_N, q = rem - srow * R_N;
    __nv_bfloat16* ob = out + ((long long)(l * R_N + q) * T * R_f + srow) * BKC;
    float v[VPT];
    float m = 0.0f;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int i = (k * TPB + threadIdx.x);  // coalesced
      v[k] = (i < n) ? float(x[i]) : 0.0f;
      m = fmaxf(m, fabsf(v[k]));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    float mm = red[0];
#pragma unroll
    for (int w = 1; w < TPB / 32; ++w) mm = fmaxf(mm, red[w]);
    int e = 0;
    if (mm > 0.0f) {
      frexpf(mm, &e);  // mm = f 2^e, f in [0.5, 1): |x| < 2^e
      if (BAL) e += 1;  // balanced digits: |x| < 2^(e-1)
    }
    if (threadIdx.x == 0) expo[row] = e;
    // 2^(8-e) as two exact multiplies by normal powers of two (as the convolution's epilogue)
    const int k1 = (8 - e) / 2, k2 = (8 - e) - k1;
    const float sc1 = __int_as_float((127 + k1) << 23), sc2 = __int_as_float((127 + k2) << 23);
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int i = k * TPB + threadIdx.x;
      if (i >= n) continue;
      __nv_bfloat16* o = ob + (long long)(i / BKC) * R_f * BKC + (i % BKC);
      float a = (v[k] * sc1) * sc2;  // |a| < 256 (balanced: 128)
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        const float d = rintf(a);  // digit s_j: |s_0| <= 256 (balanced: 128), |s_j| <= 128
        a = (a - d) * 256.0f;      // exact
        o[j * slice_stride] = __float2bfloat16_rn(d);
      }
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
  int raster;              // rows mode: 256-row blocks whose pairs sweep the column tiles together
  const int* qlist;        // the kernel terms of blockIdx.y (NULL: term blockIdx.y)
  // E_H: the last n_virtual rows of the grid are lag rows (their W slice
  // slots hold lag rows, not the term's W): they write their Gram blocks to
  // Gv [3][n_virtual][M][M] (float64) and add nothing to E_H
  void* Gv;
  int n_virtual;
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
template <class F>
__device__ __forceinline__ void issue_stage(const CUtensorMap* mapA, const CUtensorMap* mapB, const Args& g,
                                            uint32_t sbase, uint32_t fullbar_cluster, int tt, int T, int q, int r0,
                                            int sb0) {
  const int l = tt / T, t = tt % T;
  const uint32_t stage = sbase + (tt % F::STAGES) * F::STAGE_BYTES;
  // all slices of each operand tile in one copy: A dims (cell, r, t, l, slice),
  // B dims (cell, s, t, l*R_N + q, slice); rows past R_f read as zeros
  tma_load_5d(stage, mapA, r0, t, l, fullbar_cluster);
  tma_load_5d(stage + F::NS * F::A_SLICE_BYTES, mapB, sb0, t, l * g.R_N + q, fullbar_cluster);
}

// the slice-pair products of one chunk for the CTA pair (M = 256, N = 128):
// pair (a, b) goes to accumulator min(a + b, NACC - 1); the first MMA into
// each accumulator of a group is (0, g) at k-step 0
template <class F>
__device__ __forceinline__ void issue_mmas(uint32_t stage, uint32_t tacc, uint32_t accumulate) {
  constexpr uint32_t idesc = umma::idesc_bf16_f32(2 * BM, BN);
  const uint32_t a0 = stage, b0 = stage + F::NS * F::A_SLICE_BYTES;
#pragma unroll
  for (int a = 0; a < F::NS; ++a) {
#pragma unroll
    for (int b = 0; a + b < F::NS; ++b) {
      const int grp = a + b < F::NACC - 1 ? a + b : F::NACC - 1;
#pragma unroll
      for (int kk = 0; kk < F::K_STEPS; ++kk) {
        const uint64_t ad = desc_k<F::ROW>(a0 + a * F::A_SLICE_BYTES + kk * 32);
        const uint64_t bd = desc_k<F::ROW>(b0 + b * F::B_SLICE_BYTES + kk * 32);
        const uint32_t acc = (a == 0 && b == grp && kk == 0) ? accumulate : 1u;
        umma::mma_bf16_pair(tacc + grp * BN, ad, bd, idesc, acc);
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
// 32 (w / 4)..), warp 16 issues the pair's MMAs (even CTA) and warp 17 drives
// the copies (both CTAs): with copies and MMAs in one thread, the copy issue
// and the waits for a stage to empty kept the MMA queue from staying full
// (measured: 42% of that thread's time outside MMA issue).  GROUP consecutive chunks (256
// or 512 cells) accumulate before each readout (S_0 and S_1 stay exact).
// Barriers: full[stage] (even CTA: both halves landed), sfree[stage] (both
// CTAs: the MMAs reading a stage finished), done (both CTAs: a group of
// chunks accumulated), freeb (even CTA: the 32 reader warps of the pair
// took the accumulators out of TMEM).
// GOUT (CPC_FP64_TC): the readers fold in float64 and write G (both
// triangles); there is no product over axes and no E_H or row sum here.
// register cap: each of the SM's four sub-partitions holds 16K registers and
// a block's warps are spread over them, so the 18 warps put 5 on two of them:
// at most 16384 / (5 x 32) = 102 registers per thread, 96 in steps of 8 (104
// and 120 did not launch with 17 warps); with the cap ptxas spills 40-108
// bytes instead of the 144-168 bytes it chose under __launch_bounds__
template <class F, bool GOUT>
__global__ void __cluster_dims__(2, 1, 1) __maxnreg__(96)
gemm3_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Args g) {
  static_assert(GOUT ? F::NACC == 4 : F::NACC == 3, "TMEM columns: accumulators (+ product over axes)");
  constexpr int GROUP = F::GROUP;
  constexpr int NT = THREADS;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = umma::smem_u32(smem_raw);
  const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
  uint8_t* smem = smem_raw + pad;
  const uint32_t sbase = raw + pad;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + F::STAGES * F::STAGE_BYTES);  // [F::STAGES]
  uint64_t* sfree = full + F::STAGES;                                                // [F::STAGES]
  uint64_t* done = sfree + F::STAGES;                                                // [1]
  uint64_t* freeb = done + 1;                                                     // [1]
  uint32_t* tmem_ptr = reinterpret_cast<uint32_t*>(freeb + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_ptr + 1);
  double* col_c = reinterpret_cast<double*>(smem + F::STAGES * F::STAGE_BYTES + 256);  // [BN]
  int* col_e = reinterpret_cast<int*>(col_c + BN);                                 // [3][BN]
  double* row_q = reinterpret_cast<double*>(col_e + 3 * BN);                       // [4][BM]
  __shared__ double red[NT / 32];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = umma::cluster_ctarank();
  const int q = g.qlist ? __ldg(g.qlist + blockIdx.y) : int(blockIdx.y);
  const int vrow = int(blockIdx.y) - (int(gridDim.y) - g.n_virtual);  // >= 0: a lag row
  const bool virt = !g.rows_mode && vrow >= 0;
  const int n_ct = (g.Ns + BN - 1) / BN;
  const int pair = blockIdx.x >> 1;
  int ct, r0;
  if (g.rows_mode) {
    // rectangular 256-row x 128-column pair tiles, rastered in groups of
    // `raster` row blocks: consecutive pairs take the rows of one group for a
    // column tile, then the next column tile, so the pairs in flight share both
    // their row blocks and their column tiles in L2
    const int n_rp = (g.M + 2 * BM - 1) / (2 * BM);
    const int per_group = g.raster * n_ct;
    const int grp = pair / per_group, rem = pair - grp * per_group;
    const int rows_here = min(g.raster, n_rp - grp * g.raster);
    ct = rem / rows_here;
    const int rp = grp * g.raster + (rem - ct * rows_here);
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
  for (int i = tid; i < 4 * BN; i += NT) {
    const int j = i % BN, s = s0 + j;
    if (i < BN) col_c[j] = (s < g.Ns && g.c_col) ? g.c_col[s] : 0.0;
    else col_e[i - BN] = (s < g.Ns) ? g.eB[((long long)(i / BN - 1) * g.Ns + s) * g.R_N + q] : 0;
  }
  if (warp == 0) umma::tmem_alloc_pair(tmem_ptr, TMEM_COLS);
  if (tid == 32) {
    for (int i = 0; i < F::STAGES; ++i) {
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
  const int T = g.n / F::BKC, TT = 3 * T;  // chunks per axis, in all
  // chunks accumulate in TMEM in groups of up to GROUP (the last group of an
  // axis may be shorter); GA groups per axis, 3 GA in all
  const int GA = (T + GROUP - 1) / GROUP;
  const uint32_t freeb_even = umma::mapa(umma::smem_u32(freeb), 0);
  double sum = 0.0;

  if (warp == READERS + 1) {
    if (lane == 0) {
      // copies: chunk tt goes to stage tt % STAGES once the MMAs of chunk
      // tt - STAGES (the stage's previous contents) finished; both CTAs'
      // copies count on the even CTA's full barrier, which expects both halves
      for (int tt = 0; tt < TT; ++tt) {
        if (tt >= F::STAGES &&
            !wait_or_abort(&sfree[tt % F::STAGES], ((tt - F::STAGES) / F::STAGES) & 1, abort_flag))
          break;
        if (rank == 0) mbar_expect_tx(umma::smem_u32(&full[tt % F::STAGES]), 2 * F::STAGE_BYTES);
        issue_stage<F>(&mapA, &mapB, g, sbase, umma::mapa(umma::smem_u32(&full[tt % F::STAGES]), 0), tt, T, q,
                       r0, sb0);
      }
      // drain: every commit of the pair has arrived on this CTA's stage barriers
      // before the CTA can leave
      if (!*abort_flag)
        for (int tt = (TT > F::STAGES ? TT - F::STAGES : 0); tt < TT; ++tt)
          if (!wait_or_abort(&sfree[tt % F::STAGES], (tt / F::STAGES) & 1, abort_flag)) break;
    }
  } else if (warp == READERS) {
    if (lane == 0 && rank == 0) {
      // the pair's MMAs: wait for a chunk's data (and, at the start of a group,
      // for the readers to empty the accumulators), issue, commit
      for (int tt = 0; tt < TT; ++tt) {
        const int t = tt % T, gi = (tt / T) * GA + t / GROUP;  // group of this chunk
        const bool first = (t % GROUP == 0), last = (t % GROUP == GROUP - 1) || (t == T - 1);
        if (!wait_or_abort(&full[tt % F::STAGES], (tt / F::STAGES) & 1, abort_flag)) break;
        if (first && gi >= 1 && !wait_or_abort(freeb, (gi - 1) & 1, abort_flag)) break;
        umma::fence_after();
        issue_mmas<F>(sbase + (tt % F::STAGES) * F::STAGE_BYTES, tbase, first ? 0u : 1u);
        umma::mma_commit_pair(&sfree[tt % F::STAGES]);
        if (last) umma::mma_commit_pair(done);
      }
    }
  } else {
    const int quad = warp & 3, part = warp >> 2;
    const int r = r0 + 32 * quad + lane;  // this thread's row and TMEM lane
    const uint32_t lane_base = tbase + (static_cast<uint32_t>(32 * quad) << 16) + part * BNW;
    const int sh0 = s0 + part * BNW;  // first column of this warp
    // float32 form: running sum of an axis as an unevaluated pair tot + lo
    // (TwoSum per fold); |lo| stays near 2^-24 |tot|, so lo is kept in bf16
    // (two per register): its own rounding is then below 2^-32 |tot|.
    // CPC_FP64_TC: an unevaluated float pair hi + lo per entry (TwoSum of each
    // of the four group sums into hi, the rounding errors summed in lo: about
    // 48 bits, and float32 arithmetic; this GPU's float64 rate made a float64
    // fold as slow as the MMAs it folds).
    float tot[BNW];
    __nv_bfloat162 lo[GOUT ? 1 : BNW / 2];
    float lo32[GOUT ? BNW : 1];
#pragma unroll
    for (int j = 0; j < BNW; ++j) {
      tot[j] = 0.0f;
      if constexpr (GOUT) lo32[j] = 0.0f;
    }
    if constexpr (!GOUT) {
#pragma unroll
      for (int j = 0; j < BNW / 2; ++j) lo[j] = __float2bfloat162_rn(0.0f);
    }
    double row = 0.0;
    bool ok = true;
    for (int gi = 0; gi < 3 * GA && ok; ++gi) {
      if (!wait_or_abort(done, gi & 1, abort_flag)) { ok = false; break; }
      umma::fence_after();
#pragma unroll
      for (int cb = 0; cb < BNW / 8; ++cb) {
        float v0[8], v1[8], v2[8], v3[8];
        const uint32_t col = cb * 8;
        umma::tmem_ld8(lane_base + col, v0);
        umma::tmem_ld8(lane_base + col + BN, v1);
        umma::tmem_ld8(lane_base + col + 2 * BN, v2);
        if constexpr (F::NACC > 3) umma::tmem_ld8(lane_base + col + 3 * BN, v3);
        umma::tmem_ld_wait();
        if constexpr (GOUT) {
          // weighted slices: the four sums already carry their weights
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float& t = tot[cb * 8 + j];
            float e = 0.0f;
            const float vs[4] = {v0[j], v1[j], v2[j], v3[j]};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float sm = t + vs[k], bb = sm - t;
              e += (t - (sm - bb)) + (vs[k] - bb);
              t = sm;
            }
            lo32[cb * 8 + j] += e;
          }
        } else {
          // two columns at a time in paired float32 instructions (the same
          // roundings as the scalar fold: y - x is written fma(x, -1, y))
          const float2 k8 = make_float2(1.0f / 256.0f, 1.0f / 256.0f);
          const float2 k16 = make_float2(1.0f / 65536.0f, 1.0f / 65536.0f);
          const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const float2 v = __ffma2_rn(make_float2(v2[j], v2[j + 1]), k16,
                                        __ffma2_rn(make_float2(v1[j], v1[j + 1]), k8, make_float2(v0[j], v0[j + 1])));
            const float2 t = make_float2(tot[cb * 8 + j], tot[cb * 8 + j + 1]);
            const float2 sm = __fadd2_rn(t, v);
            const float2 bb = __ffma2_rn(t, m1, sm);                                   // sm - t
            const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, sm), m1, t),      // t - (sm - bb)
                                        __ffma2_rn(bb, m1, v));                         // + (v - bb)
            tot[cb * 8 + j] = sm.x;
            tot[cb * 8 + j + 1] = sm.y;
            __nv_bfloat162& L = lo[(cb * 8 + j) / 2];
            L = __float22bfloat162_rn(__fadd2_rn(__bfloat1622float2(L), e));
          }
        }
      }
      umma::fence_before();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive_cluster(freeb_even);
      if (gi % GA == GA - 1) {
        // axis l finished: G_l = 2^(e_r + e_s - 16) (sum of the folds)
        const int l = gi / GA;
        const int er = (r < g.M) ? g.eA[l * g.M + r] : 0;
        if constexpr (GOUT) {
#pragma unroll
          for (int j = 0; j < BNW; ++j) {
            const int s = sh0 + j;
            const int es = col_e[l * BN + part * BNW + j];
            const double Gv = ldexp(double(tot[j]) + double(lo32[j]), er + es - 16);
            tot[j] = 0.0f;
            lo32[j] = 0.0f;
            if (r < g.M && s < g.Ns && (!diag || r <= s)) {
              double* Gq = virt ? static_cast<double*>(g.Gv) + ((size_t)l * g.n_virtual + vrow) * (size_t)g.M * g.M
                                : g.G + ((size_t)l * g.R_N + q) * (size_t)g.M * g.M;
              Gq[(size_t)r * g.M + s] = Gv;
              Gq[(size_t)s * g.M + r] = Gv;
            }
          }
        } else {
          // the running product over axes lives in TMEM columns PROD_COL.. between axes
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
              if (in && (virt || g.G)) {  // one store path (a second one costs registers)
                double* Gq = virt ? static_cast<double*>(g.Gv) + ((size_t)l * g.n_virtual + vrow) * (size_t)g.M * g.M
                                  : g.G + ((size_t)l * g.R_N + q) * (size_t)g.M * g.M;
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
    }
    if (!GOUT) {
      if (g.rows_mode) row_q[part * BM + 32 * quad + lane] = ok ? row : 0.0;
      else if (ok && r < g.M) sum = g.c[r] * row;
    }
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) red[warp] = sum;
  umma::fence_before();
  __syncthreads();
  if (GOUT) {
    if (tid == 0 && *abort_flag) atomicExch(g.status, 1);
  } else if (g.rows_mode) {
    // row sums of this CTA's 128 rows over the tile's 128 columns
    if (tid < BM && r0 + tid < g.M)
      g.partial[((size_t)q * n_ct + ct) * g.M + r0 + tid] =
          row_q[tid] + row_q[BM + tid] + row_q[2 * BM + tid] + row_q[3 * BM + tid];
    if (tid == 0 && *abort_flag) atomicExch(g.status, 1);
  } else if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    if (!virt) g.partial[(size_t)q * gridDim.x + blockIdx.x] = s;
    if (*abort_flag) atomicExch(g.status, 1);
  }
  umma::cluster_sync();  // neither CTA leaves (or frees TMEM) while the pair still works
  if (warp == 0) {
    umma::fence_after();
    umma::tmem_dealloc_pair(tbase, TMEM_COLS);
  }
}

// BAL: balanced digits (the W operand of the float32 form)
template <typename TS, class F, bool BAL>
int launch_slice(const TS* src, long long rows, int n, int R_f, int R_N, __nv_bfloat16* out, long long slice_stride,
                 int* expo, cudaStream_t s, const int* qmap = nullptr, int n_qmap = 1, int R_N_src = 1) {
  const unsigned grid = (unsigned)std::min<long long>(rows, 1 << 20);
  const int slot = timing_begin("slice_rows_kernel", s);
#define CPC_SLICE(VPT, TPB)                                                                                    \
  slice_rows_kernel<TS, VPT, F, TPB, BAL><<<grid, TPB, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo, \
                                                                qmap, n_qmap, R_N_src)
  switch (n) {
    case 128: CPC_SLICE(1, 256); break;
    case 256: CPC_SLICE(1, 256); break;
    case 512: CPC_SLICE(2, 256); break;
    case 1024: CPC_SLICE(4, 256); break;
    case 2048: CPC_SLICE(8, 256); break;
    case 4096: CPC_SLICE(16, 256); break;
    case 8192: CPC_SLICE(32, 256); break;
    default:
      timing_end(slot, s);
      return fail(CPC_ERR_UNSUPPORTED, "tensor-core contraction: n must be a power of two in [128, 8192]");
  }
#undef CPC_SLICE
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("slice_rows_kernel");
  return CPC_OK;
}

// CPC_FP64_TC slicing in two streaming passes (the per-row reduction and the
// digits in one kernel left a CTA per row waiting on its loads).
// Pass 1: expo[row] = e with 2^e > max|x| over the row (frexp convention),
// from the largest biased exponent field of the row's float64 values
// (0 for a row of zeros or subnormals); 256 threads per row, rows grid-strided.
__global__ void __launch_bounds__(256) row_exponent64_kernel(const double* __restrict__ src, long long rows, int n,
                                                             int* __restrict__ expo) {
  __shared__ int red[8];
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const double2* x = reinterpret_cast<const double2*>(src + row * n);
    int m = 0;
    for (int i = threadIdx.x; i < n / 2; i += 256) {
      const double2 v = x[i];
      m = max(m, max(int((__double_as_longlong(v.x) >> 52) & 0x7FF), int((__double_as_longlong(v.y) >> 52) & 0x7FF)));
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      int mm = red[0];
      for (int w = 1; w < 8; ++w) mm = max(mm, red[w]);
      expo[row] = row_exponent64(mm);
    }
    __syncthreads();
  }
}

// Pass 2: the five weighted digits t_k = s_k 2^(-8k) of each float64 value,
// by integer arithmetic on its bit pattern (the float64 pipe of this GPU is
// slow): A = |x| 2^(40-e) rounded to an integer (half up; |x 2^(40-e) - A|
// <= 1/2, i.e. 2^-41 of 2^e), split into balanced base-256 digits s_4..s_1 in
// [-128, 127] and the leading s_0 in [0, 256], all with the sign of x (values
// below the float64 normal range count as zero).  A block per row (rows
// grid-strided, the row's place in the layout found once), two neighbouring
// cells per thread and step (one 4-byte store per slice); the output layout
// is slice_rows_kernel's.
template <int BKC>
__global__ void __launch_bounds__(256) slice64_kernel(const double* __restrict__ src, long long rows, int n, int R_f,
                                                      int R_N, __nv_bfloat16* __restrict__ out, long long slice_stride,
                                                      const int* __restrict__ expo) {
  static_assert(BKC == kSlice64Cells, "the slice layout's chunk");
  const int T = n / BKC;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    // the row's place in the chunk-blocked layout, once per row
    const long long per_l = (long long)R_f * R_N;
    const int l = (int)(row / per_l);
    const int rem = (int)(row - l * per_l);
    const int srow = rem / R_N, q = rem - srow * R_N;
    const int e = expo[row];
    const double2* x = reinterpret_cast<const double2*>(src + row * n);
    __nv_bfloat16* ob = out + ((long long)(l * R_N + q) * T * R_f + srow) * BKC;
    for (int p = threadIdx.x; p < n / 2; p += 256) {
      const int i = 2 * p;  // even cell: the pair stays in one chunk
      const double2 v = x[p];
      slice64_pair(v.x, v.y, e, ob + (i / BKC) * (long long)R_f * BKC + (i % BKC), slice_stride);
    }
  }
}

int launch_slice64(const double* src, long long rows, int n, int R_f, int R_N, __nv_bfloat16* out,
                   long long slice_stride, int* expo, cudaStream_t s) {
  const int slot = timing_begin("slice_rows_kernel", s);
  const unsigned g1 = (unsigned)std::min<long long>(rows, 152LL * 8 * 4);
  row_exponent64_kernel<<<g1, 256, 0, s>>>(src, rows, n, expo);
  const unsigned g2 = (unsigned)std::min<long long>(rows, 152LL * 8 * 4);
  slice64_kernel<Form64::BKC><<<g2, 256, 0, s>>>(src, rows, n, R_f, R_N, out, slice_stride, expo);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("slice64_kernel");
  return CPC_OK;
}

// E_H from the float64 convolution matrices (CPC_FP64_TC): block (r, q) sums
// (1 or 2) c_s prod_l G_l[q][r][s] over s >= r in a fixed order, times c_r.
__global__ void __launch_bounds__(128) eh_from_g_kernel(const double* __restrict__ G, const double* __restrict__ c,
                                                        int R_f, int R_N, double* __restrict__ partial) {
  __shared__ double red[4];
  const int r = blockIdx.x, q = blockIdx.y;
  const size_t plane = (size_t)R_f * R_f, axis = (size_t)R_N * plane;
  const double* g0 = G + (size_t)q * plane + (size_t)r * R_f;
  double acc = 0.0;
  for (int s = r + threadIdx.x; s < R_f; s += blockDim.x)
    acc += (s == r ? 1.0 : 2.0) * c[s] * (g0[s] * g0[axis + s] * g0[2 * axis + s]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) partial[(size_t)q * R_f + r] = c[r] * (((red[0] + red[1]) + red[2]) + red[3]);
}

}  // namespace tc

// one partial per CTA: 2 CTAs per pair tile of the symmetric tiling and kernel term
size_t tc_partials(int R_f, int R_N) {
  return size_t(2) * tc::eh_pair_tiles((R_f + tc::BN - 1) / tc::BN) * R_N;
}
// CPC_FP64_TC: one partial per row and kernel term (eh_from_g_kernel)
size_t tc64_partials(int R_f, int R_N) { return size_t(R_f) * R_N; }

// n a multiple of 128 (the convolution that writes the W slices needs n >= 128)
bool tc_supported(const cpc_kernel* P) { return P->n >= 128 && P->n % 128 == 0; }

namespace {
// workspace of the tensor-core contraction of M A rows against Ns R_N W rows:
// A slices, row exponents of A and W, status word, (CPC_FP64_TC: the float64
// convolution matrices G,) then the W slices (each 256-aligned)
struct TcLayout {
  size_t a, b;  // slice elements of A and W (all slices, 3 axes)
  size_t off_ea, off_eb, off_status, off_g, off_b, off_v, total;
};
TcLayout tc_layout(const cpc_kernel* P, int M, int Ns, int ns = 3, bool with_g = false) {
  TcLayout L;
  L.a = size_t(ns) * 3 * M * P->n;
  L.b = size_t(ns) * 3 * size_t(Ns) * P->R_N * P->n;
  L.off_ea = align256(2 * L.a);
  L.off_eb = L.off_ea + align256(4 * size_t(3) * M);
  L.off_status = L.off_eb + align256(4 * size_t(3) * Ns * P->R_N);
  L.off_g = L.off_status + 256;
  L.off_b = L.off_g + (with_g ? align256(sizeof(double) * 3 * size_t(P->R_N) * M * M) : 0);
  // (CPC_FP64_TC: then the lag rows' Gram matrices [3][kMaxLags][M][M])
  L.off_v = L.off_b + align256(2 * L.b);
  L.total = L.off_v + (with_g ? align256(sizeof(double) * 3 * kMaxLags * size_t(M) * M) : 0);
  return L;
}
}  // namespace

size_t tc_workspace(const cpc_kernel* P, int R_f) { return tc_layout(P, R_f, R_f).total; }
size_t tc64_workspace(const cpc_kernel* P, int R_f) { return tc_layout(P, R_f, R_f, tc::Form64::NS, true).total; }
size_t tc_rows_workspace(const cpc_kernel* P, int M, int Ns) { return tc_layout(P, M, Ns).total; }
size_t tc_rows_groups(const cpc_kernel* P, int Ns) { return size_t((Ns + tc::BN - 1) / tc::BN) * P->R_N; }

// status (int) of the tc workspace
int* tc_status_ptr(const cpc_kernel* P, int R_f, void* ws) {
  return reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + tc_layout(P, R_f, R_f).off_status);
}
int* tc64_status_ptr(const cpc_kernel* P, int R_f, void* ws) {
  return reinterpret_cast<int*>(static_cast<unsigned char*>(ws) + tc_layout(P, R_f, R_f, tc::Form64::NS, true).off_status);
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
// tensor maps of the chunk-blocked slices and the launch
template <class F, bool GOUT>
int launch_tc_kernel(const cpc_kernel* P, int M, int Ns, const TcLayout& L, unsigned char* w, const double* c,
                     const double* c_col, double* G, double* partial, cudaStream_t s, int rows_mode, int raster,
                     const int* qlist = nullptr, int n_q = -1, void* Gv = nullptr, int n_virtual = 0) {
  const int n = P->n, R_N = P->R_N;
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(w);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(w + L.off_b);
  int* eA = reinterpret_cast<int*>(w + L.off_ea);
  int* eB = reinterpret_cast<int*>(w + L.off_eb);
  int* status = reinterpret_cast<int*>(w + L.off_status);
  EncodeTiledFn enc;
  int st = encode_fn(&enc);
  if (st) return st;
  CUtensorMap mapA, mapB;
  const int T = n / F::BKC;
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapSwizzle swz = F::ROW == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  const cuuint64_t row = F::ROW;
  {
    // [slice NS][l 3][t T][r M][BKC cells]
    const cuuint64_t dims[5] = {(cuuint64_t)F::BKC, (cuuint64_t)M, (cuuint64_t)T, 3, (cuuint64_t)F::NS};
    const cuuint64_t strides[4] = {row, row * M, row * M * T, row * M * T * 3};
    const cuuint32_t box[5] = {(cuuint32_t)F::BKC, tc::BM, 1, 1, (cuuint32_t)F::NS};
    if (enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, As, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CPC_ERR_CUDA, "tensor map for the U slices");
  }
  {
    // [slice NS][l*R_N + q][t T][s Ns][BKC cells]
    const cuuint64_t dims[5] = {(cuuint64_t)F::BKC, (cuuint64_t)Ns, (cuuint64_t)T, (cuuint64_t)3 * R_N,
                                (cuuint64_t)F::NS};
    const cuuint64_t strides[4] = {row, row * Ns, row * Ns * T, row * Ns * T * 3 * R_N};
    const cuuint32_t box[5] = {(cuuint32_t)F::BKC, tc::BNH, 1, 1, (cuuint32_t)F::NS};
    if (enc(&mapB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, Bs, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(CPC_ERR_CUDA, "tensor map for the V_H factor slices");
  }
  const int n_rp = (M + 2 * tc::BM - 1) / (2 * tc::BM), n_ct = (Ns + tc::BN - 1) / tc::BN;
  const long long gx = rows_mode ? 2LL * n_rp * n_ct : 2LL * tc::eh_pair_tiles(n_ct);
  if (!qlist) n_q = R_N;
  if (gx > 0x7fffffffLL || n_q > 65535) return fail(CPC_ERR_UNSUPPORTED, "tensor-core contraction: grid too large");
  if (n_q <= 0) return CPC_OK;
  dim3 grid((unsigned)gx, n_q);  // clusters of 2 along x
  tc::Args args{eA,     eB, M,      Ns, R_N, n, rows_mode, c, c_col, partial, G, status,
                std::max(1, std::min(raster, n_rp)), qlist, Gv, n_virtual};
  auto kern = tc::gemm3_tc_kernel<F, GOUT>;
  CPC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(F::SMEM)));
  {
    // the block must fit the register file at this kernel's register count
    cudaFuncAttributes fa;
    CPC_CUDA(cudaFuncGetAttributes(&fa, kern));
    if (fa.maxThreadsPerBlock < tc::THREADS)
      return fail(CPC_ERR_CUDA, "gemm3_tc_kernel: " + std::to_string(fa.numRegs) + " registers per thread allow " +
                                    std::to_string(fa.maxThreadsPerBlock) + " threads per block, the kernel needs " +
                                    std::to_string(tc::THREADS));
  }
  const int slot = timing_begin("gemm3_tc_kernel", s);
  kern<<<grid, tc::THREADS, F::SMEM, s>>>(mapA, mapB, args);
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("gemm3_tc_kernel");
  return CPC_OK;
}

// float32 form: slices (unless the convolution already wrote W's), tensor maps and the launch
template <class F>
int launch_tc_form(const cpc_kernel* P, int M, int Ns, const double* U, const float* W, const double* c,
                   const double* c_col, double* G, double* partial, void* ws, cudaStream_t s, bool w_sliced,
                   int rows_mode, int raster, const int* qlist = nullptr, int n_q = -1, const int* wmap = nullptr,
                   int n_wmap = 1, int R_N_src = 1, void* Gv = nullptr, int n_virtual = 0) {
  const int n = P->n, R_N = P->R_N;
  const TcLayout L = tc_layout(P, M, Ns);
  unsigned char* w = static_cast<unsigned char*>(ws);
  CPC_CUDA(cudaMemsetAsync(w + L.off_status, 0, sizeof(int), s));
  int st0 = tc::launch_slice<double, F, false>(U, 3LL * M, n, M, 1, reinterpret_cast<__nv_bfloat16*>(w),
                                               (long long)(L.a / 3), reinterpret_cast<int*>(w + L.off_ea), s);
  if (st0) return st0;
  if (!w_sliced) {  // else the convolution already wrote them (convolve_operands32_sliced)
    st0 = tc::launch_slice<float, F, F::BAL>(W, 3LL * Ns * R_N, n, Ns, R_N,
                                             reinterpret_cast<__nv_bfloat16*>(w + L.off_b), (long long)(L.b / 3),
                                             reinterpret_cast<int*>(w + L.off_eb), s, wmap, n_wmap, R_N_src);
    if (st0) return st0;
  }
  return launch_tc_kernel<F, false>(P, M, Ns, L, w, c, c_col, G, partial, s, rows_mode, raster, qlist, n_q, Gv,
                                    n_virtual);
}
int launch_tc(const cpc_kernel* P, int M, int Ns, const double* U, const float* W, const double* c,
              const double* c_col, double* G, double* partial, void* ws, cudaStream_t s, bool w_sliced,
              int rows_mode, int raster = 1, const int* qlist = nullptr, int n_q = -1, void* Gv = nullptr,
              int n_virtual = 0) {
  return launch_tc_form<tc::Form32>(P, M, Ns, U, W, c, c_col, G, partial, ws, s, w_sliced, rows_mode, raster, qlist,
                                    n_q, nullptr, 1, 1, Gv, n_virtual);
}
}  // namespace

int launch_eh_tc(const cpc_kernel* P, int R_f, const double* U, const float* W, const double* c, double* G,
                 double* partial, void* ws, cudaStream_t s, bool w_sliced, const int* qlist, int n_q, double* Gv,
                 int n_virtual) {
  // with a term list the other terms' partial slots stay zero
  if (qlist) CPC_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * tc_partials(R_f, P->R_N), s));
  return launch_tc(P, R_f, R_f, U, W, c, c, G, partial, ws, s, w_sliced, 0, 1, qlist, n_q, Gv, n_virtual);
}

// CPC_FP64_TC: five weighted slices of the float64 U and W, the convolution
// matrices in float64 (into G, or the workspace's G when G is NULL), then
// partial[q R_f + r] = c_r sum_{s >= r} (1 or 2) c_s prod_l G_l[q][r][s]
SliceRows tc64_w_slices(const cpc_kernel* P, int R_f, void* ws) {
  const TcLayout L = tc_layout(P, R_f, R_f, tc::Form64::NS, true);
  unsigned char* w = static_cast<unsigned char*>(ws);
  return SliceRows{reinterpret_cast<__nv_bfloat16*>(w + L.off_b), (long long)(L.b / tc::Form64::NS),
                   reinterpret_cast<int*>(w + L.off_eb), R_f};
}

int launch_eh_tc64(const cpc_kernel* P, int R_f, const double* U, const double* W, const double* c, double* G,
                   double* partial, void* ws, cudaStream_t s, bool w_sliced, const void* cheb_scratch) {
  const int n = P->n, R_N = P->R_N;
  const TcLayout L = tc_layout(P, R_f, R_f, tc::Form64::NS, true);
  unsigned char* w = static_cast<unsigned char*>(ws);
  CPC_CUDA(cudaMemsetAsync(w + L.off_status, 0, sizeof(int), s));
  int st = tc::launch_slice64(U, 3LL * R_f, n, R_f, 1, reinterpret_cast<__nv_bfloat16*>(w),
                              (long long)(L.a / tc::Form64::NS), reinterpret_cast<int*>(w + L.off_ea), s);
  if (st) return st;
  if (!w_sliced) {  // else the convolution already wrote them
    st = tc::launch_slice64(W, 3LL * R_f * R_N, n, R_f, R_N, reinterpret_cast<__nv_bfloat16*>(w + L.off_b),
                            (long long)(L.b / tc::Form64::NS), reinterpret_cast<int*>(w + L.off_eb), s);
    if (st) return st;
  }
  double* Gd = G ? G : reinterpret_cast<double*>(w + L.off_g);
  int n_q = P->R_N, n_v = 0;
  const int* qlist = cheb_scratch ? eh_terms(P, 1, &n_q, &n_v) : nullptr;
  double* Gv = reinterpret_cast<double*>(w + L.off_v);
  st = launch_tc_kernel<tc::Form64, true>(P, R_f, R_f, L, w, c, c, Gd, partial, s, 0, 1, qlist, n_q, Gv, n_v);
  if (st) return st;
  if (qlist) {  // the smooth terms' G from their moments, the narrow ones' from the lag Gram matrices
    long long np = 0;
    st = launch_cheb_gram(P, 1, R_f, cheb_scratch, nullptr, Gd, nullptr, &np, s);
    if (st) return st;
    st = launch_lag_gram64(P, R_f, Gv, Gd, s);
    if (st) return st;
  }
  tc::eh_from_g_kernel<<<dim3(R_f, R_N), 128, 0, s>>>(Gd, c, R_f, R_N, partial);
  CPC_LAUNCH_CHECK("eh_from_g_kernel");
  return CPC_OK;
}

// Coulomb-matrix rows: rowpart[(q * n_ct + ct) * M + r] = sum over the 128
// columns s of tile ct of c_s prod_l G_l[r][s, q] (M item factors, Ns = R_rho)
int launch_rows_tc(const cpc_kernel* P, int M, const double* U_items, int Ns, const float* W_rho,
                   const double* c_rho, double* rowpart, void* ws, cudaStream_t s, int raster, const int* wmap,
                   int n_wmap, int R_N_src) {
  return launch_tc_form<tc::Form32>(P, M, Ns, U_items, W_rho, nullptr, c_rho, nullptr, rowpart, ws, s, false, 1, raster,
                                    nullptr, -1, wmap, n_wmap, R_N_src);
}

}  // namespace cpc
