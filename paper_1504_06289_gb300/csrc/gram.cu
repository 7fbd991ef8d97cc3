// Rank-sum contractions on CUDA cores.
//
// tri_gram_kernel computes, for rows r and columns s of two CP factor sets,
//   prod(r, s) = prod_{l=1..3} sum_i A[l][r][i] * B[l][col(s)][i]
// (three Gram matrices multiplied elementwise, Sec. 2.5 Eq. scal) and reduces
// it with weights:
//   MODE_EH   : sum_{r,s} wr[r] ws[s] prod(r,s) over symmetric tile pairs,
//               one partial per CTA (E_H, and the convolution matrices
//               M_q^(l) = U^T (p_q * U) of Sec. 3.2 Eq. Factor_Mk_Conv when
//               requested);
//   MODE_ROWS : per-row sums sum_s ws[s] prod(r,s) (Coulomb matrix rows).
// Tiles are 64 x 64 with 256 threads (4 x 4 outputs each); the K dimension
// (grid cells) is staged through shared memory in chunks.  float64 form:
// float64 FMA.  float32 form: float32 products and float32 partial sums over a
// chunk, promoted to float64 once per chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "cpc_internal.h"

namespace cpc {

constexpr int TM = 64, TN = 64, TPB = 256;

template <typename TB> struct GramCfg;
template <> struct GramCfg<double> { static constexpr int KC = 16; using TC = double; };
template <> struct GramCfg<float> { static constexpr int KC = 32; using TC = float; };

enum { MODE_EH = 0, MODE_ROWS = 1 };

// Accumulate one 64x64 Gram tile of axis l into acc[4][4] (float64).
// A rows: A + r*n (double); B columns: B + (s*col_stride + col_off)*n (TB).
template <typename TB>
__device__ __forceinline__ void gram_tile(int n, int M, int N, const double* __restrict__ A, int r0,
                                          const TB* __restrict__ B, int s0, int col_stride, int col_off,
                                          double (&acc)[4][4]) {
  using C = GramCfg<TB>;
  using TC = typename C::TC;
  constexpr int KC = C::KC;
  __shared__ TC As[KC][TM + 1];
  __shared__ TC Bs[KC][TN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int i0 = 0; i0 < n; i0 += KC) {
    for (int idx = tid; idx < TM * KC; idx += TPB) {
      const int row = idx / KC, kk = idx % KC;
      const int r = r0 + row, i = i0 + kk;
      As[kk][row] = (r < M && i < n) ? TC(A[(size_t)r * n + i]) : TC(0);
      const int s = s0 + row;
      Bs[kk][row] = (s < N && i < n) ? TC(B[((size_t)s * col_stride + col_off) * n + i]) : TC(0);
    }
    __syncthreads();
    TC part[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) part[a][b] = TC(0);
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      TC av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) part[a][b] = fma(av[a], bv[b], part[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += double(part[a][b]);
    __syncthreads();
  }
}

template <typename TB, int MODE>
__global__ void __launch_bounds__(TPB)
tri_gram_kernel(int n, int M, int N, const double* __restrict__ A, long long a_axis,
                const TB* __restrict__ B, long long b_axis, int col_stride,
                const double* __restrict__ wr, const double* __restrict__ wcol, int wcol_div,
                double* __restrict__ partial, double* __restrict__ G, int tiles_per_cta) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  __shared__ double red[TPB / 32];
  if (MODE == MODE_EH) {
    // blockIdx.x: symmetric tile pair (rt <= st); blockIdx.y: kernel term q
    const int p = blockIdx.x, q = blockIdx.y;
    int st = 0;
    while ((st + 1) * (st + 2) / 2 <= p) ++st;
    const int rt = p - st * (st + 1) / 2;
    const int r0 = rt * TM, s0 = st * TN;
    double prod[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) prod[a][b] = 1.0;
    for (int l = 0; l < 3; ++l) {
      double acc[4][4];
      gram_tile<TB>(n, M, N, A + l * a_axis, r0, B + l * b_axis, s0, col_stride, q, acc);
      if (G) {
        // G[l][q][r][s] (and the mirror for off-diagonal tiles)
        double* Gq = G + ((size_t)l * gridDim.y + q) * (size_t)M * M;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = r0 + ty + 16 * a, s = s0 + tx + 16 * b;
            if (r < M && s < N) {
              Gq[(size_t)r * M + s] = acc[a][b];
              if (rt != st) Gq[(size_t)s * M + r] = acc[a][b];
            }
          }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) prod[a][b] *= acc[a][b];
    }
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int r = r0 + ty + 16 * a;
      const double w_r = (r < M) ? wr[r] : 0.0;
      double row = 0.0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int s = s0 + tx + 16 * b;
        row += ((s < N) ? wcol[s] : 0.0) * prod[a][b];
      }
      sum += w_r * row;
    }
    if (rt != st) sum *= 2.0;
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((tid & 31) == 0) red[tid >> 5] = sum;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < TPB / 32; ++w) s += red[w];
      partial[(size_t)q * gridDim.x + p] = s;
    }
  } else {
    // persistent: work unit u = (row tile u % n_rt, column group u / n_rt);
    // CTAs with neighbouring u share the group's column tiles in L2
    const int n_rt = (M + TM - 1) / TM;
    const int n_ct = (N + TN - 1) / TN;
    const int n_groups = (n_ct + tiles_per_cta - 1) / tiles_per_cta;
    for (long long u = blockIdx.x; u < (long long)n_rt * n_groups; u += gridDim.x) {
    const int rt = int(u % n_rt), grp = int(u / n_rt);
    const int r0 = rt * TM;
    double rowacc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int ct = grp * tiles_per_cta; ct < min(n_ct, (grp + 1) * tiles_per_cta); ++ct) {
      const int s0 = ct * TN;
      double prod[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) prod[a][b] = 1.0;
      for (int l = 0; l < 3; ++l) {
        double acc[4][4];
        gram_tile<TB>(n, M, N, A + l * a_axis, r0, B + l * b_axis, s0, col_stride, 0, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) prod[a][b] *= acc[a][b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int s = s0 + tx + 16 * b;
          rowacc[a] += ((s < N) ? wcol[s / wcol_div] : 0.0) * prod[a][b];
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double v = rowacc[a];
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 16);
      const int r = r0 + ty + 16 * a;
      if (tx == 0 && r < M) partial[(size_t)grp * M + r] = v;
    }
    }
  }
}

// E_H = h^3 * sum of partials, summed in a fixed order by one block; NaN when
// a device-side wait of the contraction gave up (status != 0).
__global__ void finalize_sum_kernel(const double* __restrict__ partial, long long count, double scale,
                                    double* __restrict__ out, const int* __restrict__ status = nullptr) {
  __shared__ double red[1024 / 32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < count; i += blockDim.x) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    *out = (status && *status) ? __longlong_as_double(0x7ff8000000000000LL) : scale * t;
  }
}

// J[t] = h^3 sum_{r in item t} c[r] sum_g rowpart[g][r]
__global__ void item_reduce_kernel(int n_items, const int* __restrict__ off, const double* __restrict__ c,
                                   const double* __restrict__ rowpart, int groups, int M, double scale,
                                   double* __restrict__ J, const int* __restrict__ status = nullptr,
                                   const int* __restrict__ status2 = nullptr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_items) return;
  double s = 0.0;
  const int r_lo = max(0, min(off[t], M)), r_hi = max(r_lo, min(off[t + 1], M));
  for (int r = r_lo; r < r_hi; ++r) {
    double rs = 0.0;
    for (int g = 0; g < groups; ++g) rs += rowpart[(size_t)g * M + r];
    s += c[r] * rs;
  }
  // a device-side wait of the tensor-core kernel that gave up makes the results NaN
  const bool gave_up = (status && *status) || (status2 && *status2);
  J[t] = gave_up ? __longlong_as_double(0x7ff8000000000000LL) : scale * s;
}

// float32 form of the adjoint GEMM.  The K sum runs q-major (kk = (q, k')),
// so the A tile Bl[m][k'] for one q is read along k' (contiguous in G); A is
// formed as float(G1 G2) times float32 coefficients cached in shared memory;
// each K chunk of 32 is summed in float32 and folded into a compensated
// float32 total per output.  Tile TM m x TN i with RT x CT outputs per thread
// (rows RT ty.., columns CT tx..).  Software pipeline: while chunk c is
// multiplied out of one shared-memory buffer, the W tile of chunk c+1 lands in
// the other by cp.async and its G values wait in registers.
namespace adj32 {
constexpr int KC = 32, THREADS = 256;
constexpr int TM = 40, TN = 128, RT = 5, CT = 4;  // 40 rows: R_f = 200 splits without a ragged tile
constexpr int MAXRF = 1024;                       // coefficients cached in shared memory
constexpr int AE = (TM * KC + THREADS - 1) / THREADS;    // A elements per thread
constexpr int BE = (KC * TN / 4 + THREADS - 1) / THREADS;  // B float4 per thread
static_assert((TM / RT) * (TN / CT) == THREADS, "thread tiling");

__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(sdst))),
               "l"(gsrc));
}

__global__ void __launch_bounds__(THREADS)
adjoint32_kernel(int n, int R_f, int R_N, const double* __restrict__ c, const double* __restrict__ G,
                 const float* __restrict__ W, float scale2h3, double* __restrict__ dU) {
  __shared__ float As[2][KC][TM + 1];  // written along kk (padded: no bank conflicts)
  __shared__ __align__(16) float Bs[2][KC][TN];
  __shared__ float cf[MAXRF];
  const int l = blockIdx.z;
  const int m0 = blockIdx.y * TM, i0 = blockIdx.x * TN;
  const int tid = threadIdx.x;
  constexpr int NTX = TN / CT;
  const int tx = tid % NTX, ty = tid / NTX;
  const int l1 = (l + 1) % 3, l2 = (l + 2) % 3;
  const size_t GM = (size_t)R_f * R_f;
  const float* Wl = W + (size_t)l * R_f * R_N * n;
  for (int k = tid; k < R_f && k < MAXRF; k += THREADS) cf[k] = float(c[k]);
  const int NKP = (R_f + KC - 1) / KC, NCH = R_N * NKP;

  double g1[AE], g2[AE];
  // raw G values of chunk ch into registers (zero outside)
  auto load_a = [&](int ch) {
    const int q = ch / NKP, kp0 = (ch % NKP) * KC;
    const double* G1 = G + ((size_t)l1 * R_N + q) * GM;
    const double* G2 = G + ((size_t)l2 * R_N + q) * GM;
#pragma unroll
    for (int e = 0; e < AE; ++e) {
      const int idx = tid + e * THREADS;
      const int row = idx / KC, kk = idx % KC;
      const int m = m0 + row, kp = kp0 + kk;
      const bool ok = idx < TM * KC && m < R_f && kp < R_f;
      const size_t gi = (size_t)m * R_f + kp;
      g1[e] = ok ? G1[gi] : 0.0;
      g2[e] = ok ? G2[gi] : 0.0;
    }
  };
  // A tile of chunk ch from the registers: As[buf][kk][row] = 2 h^3 c_m c_k' G1 G2
  auto store_a = [&](int ch, int buf) {
    const int kp0 = (ch % NKP) * KC;
#pragma unroll
    for (int e = 0; e < AE; ++e) {
      const int idx = tid + e * THREADS;
      if (idx >= TM * KC) break;
      const int row = idx / KC, kk = idx % KC;
      const int m = m0 + row, kp = kp0 + kk;
      As[buf][kk][row] = (m < R_f && kp < R_f) ? (scale2h3 * cf[m] * cf[kp]) * float(g1[e] * g2[e]) : 0.0f;
    }
  };
  // W tile of chunk ch: rows k' R_N + q, columns i0.. (cp.async where whole, zeros or scalars elsewhere)
  auto load_b = [&](int ch, int buf) {
    const int q = ch / NKP, kp0 = (ch % NKP) * KC;
#pragma unroll
    for (int e = 0; e < BE; ++e) {
      const int idx = tid + e * THREADS;
      if (idx >= KC * TN / 4) break;
      const int kk = idx / (TN / 4), c4 = idx % (TN / 4);
      const int kp = kp0 + kk, i = i0 + 4 * c4;
      float* dst = &Bs[buf][kk][4 * c4];
      if (kp < R_f && i + 3 < n && (n & 3) == 0) {
        cp_async16(dst, Wl + ((size_t)kp * R_N + q) * n + i);
      } else {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kp < R_f) {
          const float* row = Wl + ((size_t)kp * R_N + q) * n;
          if (i < n) v.x = row[i];
          if (i + 1 < n) v.y = row[i + 1];
          if (i + 2 < n) v.z = row[i + 2];
          if (i + 3 < n) v.w = row[i + 3];
        }
        *reinterpret_cast<float4*>(dst) = v;
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  float tot[RT][CT], lo[RT][CT];
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < CT; ++b) { tot[a][b] = 0.0f; lo[a][b] = 0.0f; }
  __syncthreads();  // cf
  load_a(0);
  load_b(0, 0);
  store_a(0, 0);
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  for (int ch = 0; ch < NCH; ++ch) {
    const int buf = ch & 1;
    const bool more = ch + 1 < NCH;
    if (more) {
      load_b(ch + 1, buf ^ 1);
      load_a(ch + 1);
    }
    float part[RT][CT];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int b = 0; b < CT; ++b) part[a][b] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      float ar[RT];
#pragma unroll
      for (int a = 0; a < RT; ++a) ar[a] = As[buf][kk][RT * ty + a];
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][CT * tx]);
      const float br[CT] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int b = 0; b < CT; ++b) part[a][b] = fmaf(ar[a], br[b], part[a][b]);
    }
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int b = 0; b < CT; ++b) {
        const float t = tot[a][b], v = part[a][b], sm = t + v, bb = sm - t;
        lo[a][b] += (t - (sm - bb)) + (v - bb);
        tot[a][b] = sm;
      }
    if (more) store_a(ch + 1, buf ^ 1);
    asm volatile("cp.async.wait_all;\n" ::);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < RT; ++a) {
    const int m = m0 + RT * ty + a;
    if (m >= R_f) continue;
#pragma unroll
    for (int b = 0; b < CT; ++b) {
      const int i = i0 + CT * tx + b;
      if (i < n) dU[((size_t)l * R_f + m) * n + i] = double(tot[a][b]) + double(lo[a][b]);
    }
  }
}
}  // namespace adj32

// ---- adjoint --------------------------------------------------------------
// dU[l][m][i] = sum_{kk} Bl[m][kk] W[l][kk][i],  kk = k'*R_N + q,
// Bl[m][kk] = 2 h^3 c_m c_k' prod_{l' != l} G[l'][q][m][k'], formed while loading.
template <typename TB>
__global__ void __launch_bounds__(TPB)
adjoint_gemm_kernel(int n, int R_f, int R_N, const double* __restrict__ c, const double* __restrict__ G,
                    const TB* __restrict__ W, double scale2h3, double* __restrict__ dU) {
  using Cf = GramCfg<TB>;
  using TC = typename Cf::TC;
  constexpr int KC = Cf::KC;
  __shared__ TC As[KC][TM + 1];
  __shared__ TC Bs[KC][TN + 1];
  const int l = blockIdx.z;
  const int m0 = blockIdx.y * TM, i0 = blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int l1 = (l + 1) % 3, l2 = (l + 2) % 3;
  const size_t GM = (size_t)R_f * R_f;
  const TB* Wl = W + (size_t)l * R_f * R_N * n;
  const int K = R_f * R_N;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += KC) {
    for (int idx = tid; idx < TM * KC; idx += TPB) {
      // A tile: rows m, columns kk (kk fastest across threads for G reads along k'? keep simple)
      const int row = idx / KC, kk = idx % KC;
      const int m = m0 + row, k = k0 + kk;
      TC v = TC(0);
      if (m < R_f && k < K) {
        const int kp = k / R_N, q = k - kp * R_N;
        const size_t gi = (size_t)q * GM + (size_t)m * R_f + kp;
        v = TC(scale2h3 * c[m] * c[kp] * G[(size_t)l1 * R_N * GM + gi] * G[(size_t)l2 * R_N * GM + gi]);
      }
      As[kk][row] = v;
    }
    for (int idx = tid; idx < TN * KC; idx += TPB) {
      const int kk = idx / TN, col = idx % TN;
      const int k = k0 + kk, i = i0 + col;
      Bs[kk][col] = (k < K && i < n) ? TC(Wl[(size_t)k * n + i]) : TC(0);
    }
    __syncthreads();
    TC part[4][4] = {};
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      TC av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) part[a][b] = fma(av[a], bv[b], part[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += double(part[a][b]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int m = m0 + ty + 16 * a, i = i0 + tx + 16 * b;
      if (m < R_f && i < n) dU[((size_t)l * R_f + m) * n + i] = acc[a][b];
    }
}

// dc[m] = 2 h^3 sum_q sum_k' c_k' prod_l G[l][q][m][k']  (one warp per m)
__global__ void adjoint_coef_kernel(int R_f, int R_N, const double* __restrict__ c,
                                    const double* __restrict__ G, double scale2h3, double* __restrict__ dc) {
  const int m = blockIdx.x;
  const size_t GM = (size_t)R_f * R_f;
  double s = 0.0;
  for (int q = 0; q < R_N; ++q)
    for (int kp = threadIdx.x; kp < R_f; kp += blockDim.x) {
      const size_t gi = (size_t)q * GM + (size_t)m * R_f + kp;
      s += c[kp] * G[gi] * G[(size_t)R_N * GM + gi] * G[2 * (size_t)R_N * GM + gi];
    }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) dc[m] = scale2h3 * s;
}

// ---------------------------------------------------------------------------
size_t spectra_bytes(const cpc_kernel* P, int ncols, int precision);
int check_conv_args(const cpc_kernel* P, int R_f, const void* U, const void* W, int precision,
                    void* ws, size_t ws_bytes, const char* who);

static int tiles(int x) { return (x + TM - 1) / TM; }

size_t eh_partials(const cpc_kernel* P, int R_f) {
  const int T = tiles(R_f);
  // (the tensor-core and split forms' partials are followed by the smooth terms' ones)
  return std::max({size_t(T) * (T + 1) / 2 * P->R_N, eh32_partials(R_f, P->R_N) + cheb_gram_partials(P, R_f),
                   eh32a_partials(R_f, P->R_N),
                   tc_partials(R_f, P->R_N) + cheb_gram_partials(P, R_f) + lag_gram_partials(P, R_f),
                   tc64_partials(R_f, P->R_N)});
}

// contraction workspace: partial sums; float32 form: a float32 copy of U (CUDA-core
// kernel, n not a multiple of 128) or the bf16 slices, exponents and status word of
// the tensor-core kernel
size_t contraction_workspace(const cpc_kernel* P, int R_f, int precision) {
  size_t b = align256(sizeof(double) * eh_partials(P, R_f));
  // (float32 tensor-core form: then the lag Gram matrices [3][kMaxLags][R_f][R_f])
  if (precision == CPC_FP32)
    b += tc_supported(P) ? tc_workspace(P, R_f) + align256(sizeof(double) * 3 * kMaxLags * size_t(R_f) * R_f)
                         : eh32a_u32_bytes(P, R_f);
  if (precision == CPC_FP64_TC) b += tc64_workspace(P, R_f);
  return b;
}

// E_H from float32 spectra (Parseval contraction), partials in `partial`.
int launch_eh_spectral(const cpc_kernel* P, int R_f, const float2* spec32, const double* c, double* G,
                       double* E_H, double* partial, cudaStream_t s) {
  int st = launch_eh32(P, R_f, nullptr, nullptr, reinterpret_cast<const float*>(spec32), P->d_specw32, c, G,
                       partial, s);
  if (st) return st;
  finalize_sum_kernel<<<1, 1024, 0, s>>>(partial, (long long)eh32_partials(R_f, P->R_N), P->h * P->h * P->h, E_H);
  CPC_LAUNCH_CHECK("finalize_sum_kernel");
  return CPC_OK;
}

int launch_eh(const cpc_kernel* P, int R_f, const double* U, const double* c, const void* W,
              double* G, double* E_H, int precision, void* cws, cudaStream_t s) {
  double* partial = static_cast<double*>(cws);
  const int n = P->n;
  const int T = tiles(R_f);
  dim3 grid(T * (T + 1) / 2, P->R_N);
  const long long a_axis = (long long)R_f * n;
  const long long b_axis = (long long)R_f * P->R_N * n;
  long long count = (long long)grid.x * grid.y;
  if (precision == CPC_FP64) {
    tri_gram_kernel<double, MODE_EH><<<grid, TPB, 0, s>>>(n, R_f, R_f, U, a_axis, static_cast<const double*>(W),
                                                           b_axis, P->R_N, c, c, 1, partial, G, 0);
    CPC_LAUNCH_CHECK("tri_gram_kernel(EH)");
  } else if (precision == CPC_SPLIT) {
    int st = launch_eh32(P, R_f, U, nullptr, nullptr, nullptr, c, G, partial, s, static_cast<const double*>(W));
    if (st) return st;
    count = (long long)eh32_partials(R_f, P->R_N);
  } else if (precision == CPC_FP64_TC) {
    if (!tc_supported(P)) return fail(CPC_ERR_UNSUPPORTED, "CPC_FP64_TC needs n a multiple of 128");
    void* tws = static_cast<unsigned char*>(cws) + align256(sizeof(double) * eh_partials(P, R_f));
    int st = launch_eh_tc64(P, R_f, U, static_cast<const double*>(W), c, G, partial, tws, s);
    if (st) return st;
    finalize_sum_kernel<<<1, 1024, 0, s>>>(partial, (long long)tc64_partials(R_f, P->R_N), P->h * P->h * P->h, E_H,
                                           tc64_status_ptr(P, R_f, tws));
    CPC_LAUNCH_CHECK("finalize_sum_kernel");
    return CPC_OK;
  } else if (tc_supported(P)) {
    void* tws = static_cast<unsigned char*>(cws) + align256(sizeof(double) * eh_partials(P, R_f));
    int st = launch_eh_tc(P, R_f, U, static_cast<const float*>(W), c, G, partial, tws, s);
    if (st) return st;
    finalize_sum_kernel<<<1, 1024, 0, s>>>(partial, (long long)tc_partials(R_f, P->R_N), P->h * P->h * P->h, E_H,
                                           tc_status_ptr(P, R_f, tws));
    CPC_LAUNCH_CHECK("finalize_sum_kernel");
    return CPC_OK;
  } else {
    float* U32 = reinterpret_cast<float*>(static_cast<unsigned char*>(cws) + align256(sizeof(double) * eh_partials(P, R_f)));
    int st = launch_eh32a(P, R_f, U, static_cast<const float*>(W), c, G, partial, U32, s);
    if (st) return st;
    count = (long long)eh32a_partials(R_f, P->R_N);
  }
  finalize_sum_kernel<<<1, 1024, 0, s>>>(partial, count, P->h * P->h * P->h, E_H);
  CPC_LAUNCH_CHECK("finalize_sum_kernel");
  return CPC_OK;
}

// cp_hartree_energy after argument checks: convolution into W, then the
// spatial contraction of U with W in the form's precision.
int run_hartree_energy(const cpc_kernel* P, int R_f, const double* U, const double* c, void* W, double* G,
                       double* E_H, int precision, void* ws, cudaStream_t s) {
  void* cws = static_cast<unsigned char*>(ws) + cp_convolve_workspace(P, R_f, precision);
  void* scratch = static_cast<unsigned char*>(ws) + conv_spectra_bytes(P, R_f, precision);
  if (precision == CPC_FP32 && tc_supported(P)) {
    // the convolution writes W and, in the same pass, the W slices of the
    // tensor-core contraction (no second pass over W) for the banded and FFT
    // terms; the smooth terms' Gram matrices come from their moments
    void* X = ws;  // float32 convolution operands, in the float64-spectra part of the workspace
    int st = forward_operands32(P, 3 * R_f, U, X, s);
    if (st) return st;
    void* tws = static_cast<unsigned char*>(cws) + align256(sizeof(double) * eh_partials(P, R_f));
    __nv_bfloat16* sl;
    long long sl_stride;
    int* ex;
    tc_w_slices(P, R_f, tws, &sl, &sl_stride, &ex);
    st = convolve_operands32_sliced(P, R_f, X, static_cast<float*>(W), sl, sl_stride, ex, s, U, scratch);
    if (st) return st;
    // the lag rows of the narrow terms into the slice slots of covered terms
    st = lag_slices32(P, R_f, U, SliceRows{sl, sl_stride, ex, R_f}, s);
    if (st) return st;
    double* partial = static_cast<double*>(cws);
    double* Sv = reinterpret_cast<double*>(static_cast<unsigned char*>(tws) + tc_workspace(P, R_f));
    int n_q = P->R_N, n_v = 0;
    const int* qlist = eh_terms(P, 0, &n_q, &n_v);
    st = launch_eh_tc(P, R_f, U, static_cast<const float*>(W), c, G, partial, tws, s, true, qlist, n_q, Sv, n_v);
    if (st) return st;
    long long count = (long long)tc_partials(R_f, P->R_N), n_more = 0;
    st = launch_cheb_gram(P, 0, R_f, scratch, c, G, partial + count, &n_more, s);
    if (st) return st;
    count += n_more;
    st = launch_lag_gram(P, R_f, Sv, c, G, partial + count, &n_more, s);
    if (st) return st;
    count += n_more;
    finalize_sum_kernel<<<1, 1024, 0, s>>>(partial, count, P->h * P->h * P->h, E_H, tc_status_ptr(P, R_f, tws));
    CPC_LAUNCH_CHECK("finalize_sum_kernel");
    return CPC_OK;
  }
  if (precision == CPC_FP64_TC && tc_supported(P) && conv_slices64_supported(P)) {
    // likewise for the float64 form: the convolution writes W's five-digit
    // slices and row exponents into the contraction's workspace
    void* tws = static_cast<unsigned char*>(cws) + align256(sizeof(double) * eh_partials(P, R_f));
    const SliceRows so = tc64_w_slices(P, R_f, tws);
    int st = run_convolve(P, R_f, U, W, precision, ws, s, &so);
    if (st) return st;
    st = lag_slices64(P, R_f, U, so, s);  // the lag rows of the narrow terms
    if (st) return st;
    double* partial = static_cast<double*>(cws);
    // (with smooth or lag-covered terms, their G come from the convolution's
    // scratch and the lag rows; the contraction then takes the rest)
    st = launch_eh_tc64(P, R_f, U, static_cast<const double*>(W), c, G, partial, tws, s, true,
                        cheb_gram_active(P, 1) || P->n_lag[1] > 0 ? scratch : nullptr);
    if (st) return st;
    finalize_sum_kernel<<<1, 1024, 0, s>>>(partial, (long long)tc64_partials(R_f, P->R_N), P->h * P->h * P->h, E_H,
                                           tc64_status_ptr(P, R_f, tws));
    CPC_LAUNCH_CHECK("finalize_sum_kernel");
    return CPC_OK;
  }
  if (precision == CPC_SPLIT && cheb_gram_active(P, 1)) {
    // the split form likewise: the smooth terms' Gram matrices from the
    // moments, the others by the compensated float32 contraction
    int st = run_convolve(P, R_f, U, W, precision, ws, s);
    if (st) return st;
    double* partial = static_cast<double*>(cws);
    int n_q = P->R_N;
    const int* qlist = dense_terms(P, 1, &n_q);
    st = launch_eh32(P, R_f, U, nullptr, nullptr, nullptr, c, G, partial, s, static_cast<const double*>(W), qlist,
                     n_q);
    if (st) return st;
    long long count = (long long)eh32_partials(R_f, P->R_N), n_cheb = 0;
    st = launch_cheb_gram(P, 1, R_f, scratch, c, G, partial + count, &n_cheb, s);
    if (st) return st;
    finalize_sum_kernel<<<1, 1024, 0, s>>>(partial, count + n_cheb, P->h * P->h * P->h, E_H);
    CPC_LAUNCH_CHECK("finalize_sum_kernel");
    return CPC_OK;
  }
  int st = run_convolve(P, R_f, U, W, precision, ws, s);
  if (st) return st;
  return launch_eh(P, R_f, U, c, W, G, E_H, precision, cws, s);
}

}  // namespace cpc

using namespace cpc;

extern "C" size_t cp_hartree_energy_workspace(const cpc_kernel* P, int R_f, int precision) {
  if (!P || R_f <= 0) return 0;
  return cp_convolve_workspace(P, R_f, precision) + contraction_workspace(P, R_f, precision);
}

extern "C" int cp_hartree_energy(const cpc_kernel* P, int R_f, const double* U, const double* c, void* W,
                                 double* G, double* E_H, int precision, void* ws, size_t ws_bytes,
                                 void* stream) {
  clear_error();
  int st = check_conv_args(P, R_f, U, W, precision, ws, ws_bytes, "cp_hartree_energy");
  if (st) return st;
  if (!c || !E_H) return fail(CPC_ERR_INVALID, "cp_hartree_energy: NULL c or E_H");
  if (ws_bytes < cp_hartree_energy_workspace(P, R_f, precision))
    return fail(CPC_ERR_WORKSPACE, "cp_hartree_energy: workspace too small");
  return run_hartree_energy(P, R_f, U, c, W, G, E_H, precision, ws, static_cast<cudaStream_t>(stream));
}

extern "C" size_t cp_hartree_energy_from_factors_workspace(const cpc_kernel* P, int R_f, int precision) {
  if (!P || R_f <= 0) return 0;
  return contraction_workspace(P, R_f, precision);
}

extern "C" int cp_hartree_energy_from_factors(const cpc_kernel* P, int R_f, const double* U, const double* c,
                                              const void* W, double* G, double* E_H, int precision, void* ws,
                                              size_t ws_bytes, void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_CONV) return fail(CPC_ERR_INVALID, "cp_hartree_energy_from_factors: needs a CONV kernel");
  if (R_f <= 0 || !U || !c || !W || !E_H) return fail(CPC_ERR_INVALID, "cp_hartree_energy_from_factors: bad arguments");
  if (!known_precision(precision))
    return fail(CPC_ERR_UNSUPPORTED, "cp_hartree_energy_from_factors: precision form not implemented");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) ||
      ws_bytes < cp_hartree_energy_from_factors_workspace(P, R_f, precision))
    return fail(CPC_ERR_WORKSPACE, "cp_hartree_energy_from_factors: workspace missing, misaligned or too small");
  return launch_eh(P, R_f, U, c, W, G, E_H, precision, ws, static_cast<cudaStream_t>(stream));
}

extern "C" int cp_hartree_energy_adjoint(const cpc_kernel* P, int R_f, const double* c, const void* W,
                                         const double* G, double* dU, double* dc, int precision,
                                         void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_CONV) return fail(CPC_ERR_INVALID, "cp_hartree_energy_adjoint: needs a CONV kernel");
  if (R_f <= 0 || !c || !W || !G || !dU) return fail(CPC_ERR_INVALID, "cp_hartree_energy_adjoint: bad arguments");
  if (!known_precision(precision))
    return fail(CPC_ERR_UNSUPPORTED, "cp_hartree_energy_adjoint: precision form not implemented");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = P->n;
  const double scale = 2.0 * P->h * P->h * P->h;
  dim3 grid((n + TN - 1) / TN, tiles(R_f), 3);
  const int slot = timing_begin("adjoint_gemm_kernel", s);
  if (storage_precision(precision) == CPC_FP64) {
    adjoint_gemm_kernel<double><<<grid, TPB, 0, s>>>(n, R_f, P->R_N, c, G, static_cast<const double*>(W), scale, dU);
  } else {
    dim3 g32((n + adj32::TN - 1) / adj32::TN, (R_f + adj32::TM - 1) / adj32::TM, 3);
    adj32::adjoint32_kernel<<<g32, adj32::THREADS, 0, s>>>(n, R_f, P->R_N, c, G, static_cast<const float*>(W),
                                                          float(scale), dU);
  }
  timing_end(slot, s);
  CPC_LAUNCH_CHECK("adjoint_gemm_kernel");
  if (dc) {
    adjoint_coef_kernel<<<R_f, 32, 0, s>>>(R_f, P->R_N, c, G, scale, dc);
    CPC_LAUNCH_CHECK("adjoint_coef_kernel");
  }
  return CPC_OK;
}

// ---- Coulomb matrix ---------------------------------------------------------
// Items are flattened into one row space of n_factors item factors; the
// contraction runs as a persistent launch over (row tile, column group) work
// units, a column group being tiles_per_cta consecutive 64-column tiles of
// the R_rho R_N V_H columns.  tiles_per_cta trades the per-unit row-sum
// traffic (one partial per row per group) against load balance; the tuner
// below times the candidates on the caller's data.
namespace cpc {
// schedule parameter: CUDA-core forms, 64-column tiles per work unit (tuned over
// [4, 128]); tensor-core form, 256-row item blocks rastered together (tuned over
// [1, 32]); 8 when the caller passes 0
static const int kTilesDefault = 8, kTilesMin = 4, kTilesMax = 128;
static const int kRasterMin = 1, kRasterMax = 32;
static int coulomb_groups(int R_rho, int R_N, int tiles_per_cta) {
  const int n_ct = tiles(R_rho * R_N);
  return (n_ct + tiles_per_cta - 1) / tiles_per_cta;
}

// c_col[m R_N + q] = c_rho[m]: the coefficient of each (factor, term) column
__global__ void expand_coef_kernel(int R_rho, int R_N, const double* __restrict__ c, double* __restrict__ cq) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < R_rho * R_N) cq[m] = c[m / R_N];
}

// a view of P with one kernel term: the tensor-core rows form then takes the
// R_rho R_N columns (m, q) as factors of one term each, so that they fill its
// 128-column tiles (the product over axes is per column either way)
static cpc_kernel column_view(const cpc_kernel* P) {
  cpc_kernel Q;  // only the sizes the contraction reads; no tables
  Q.n = P->n;
  Q.b = P->b;
  Q.h = P->h;
  Q.kind = P->kind;
  Q.len = P->len;
  Q.R_N = 1;
  return Q;
}

// The tensor-core form takes the smooth kernel terms (CONV kernels with a
// Chebyshev path) from their moments: G[r][(m, q)] = sum_k m_{r,k} d_{m,q,k}
// (the identity of cheb_gram_kernel) as a second rows contraction whose
// "cells" are the kCheb moments and coefficients, zero-padded to a 128-cell
// tile; the banded and FFT terms are contracted over the n cells (their W
// rows gathered by the slicing).
static const int kMomCells = 128;
static bool coulomb_smooth(const cpc_kernel* P) { return P->kind == CPC_KERNEL_CONV && cheb_gram_active(P, 0); }
static cpc_kernel moment_view(const cpc_kernel* P) {
  cpc_kernel Q = column_view(P);
  Q.n = kMomCells;
  return Q;
}

// workspace of coulomb_contract (after the convolution's): column coefficients
// (dense, smooth), row partials of both contractions (contiguous), their
// tensor-core scratch, then the smooth terms' operand rows and moment partials
static size_t contract_bytes(const cpc_kernel* P, int n_factors, int R_rho, int precision) {
  if (precision == CPC_FP32 && tc_supported(P)) {
    const cpc_kernel Q = column_view(P);
    const int Nc = R_rho * P->R_N;
    size_t b = align256(sizeof(double) * Nc) + align256(sizeof(double) * tc_rows_groups(&Q, Nc) * n_factors) +
               tc_rows_workspace(&Q, n_factors, Nc);
    if (coulomb_smooth(P)) {
      const cpc_kernel Qm = moment_view(P);
      const int Ns = R_rho * P->n_smooth[0];
      b += align256(sizeof(double) * Ns) + align256(sizeof(double) * tc_rows_groups(&Qm, Ns) * n_factors) +
           tc_rows_workspace(&Qm, n_factors, Ns) + align256(sizeof(double) * 3 * size_t(n_factors) * kMomCells) +
           align256(sizeof(float) * 3 * size_t(Ns) * kMomCells) + cheb_moment_rows_scratch(P, 3 * n_factors);
    }
    return b;
  }
  return align256(sizeof(double) * coulomb_groups(R_rho, P->R_N, kTilesMin) * n_factors);
}

// contraction + segmented item reduction, after W_rho holds the V_H factors
// J[t] = scale sum_{r in item t} c_items[r] sum_m c_rho[m] sum_q prod_l <u_r^(l), W_rho[l][m R_N + q]>
// (cheb_scratch: the scratch of the convolution that wrote W_rho, whose
// Chebyshev coefficients the tensor-core form takes for the smooth terms;
// NULL: every term over the cells)
static int coulomb_contract(const cpc_kernel* P, int n_items, const int* off, int n_factors, const double* U_items,
                            const double* c_items, int R_rho, const double* c_rho, const void* W_rho, double* J,
                            int precision, int tiles_per_cta, double* rowpart, cudaStream_t s, double scale,
                            const void* cheb_scratch = nullptr) {
  const int n = P->n;
  const int N = R_rho * P->R_N;
  const int groups = coulomb_groups(R_rho, P->R_N, tiles_per_cta);
  const long long units = (long long)tiles(n_factors) * groups;
  const int grid = (int)std::min<long long>(units, 2LL * 152 * 4);
  const long long a_axis = (long long)n_factors * n;
  const long long b_axis = (long long)N * n;
  int st = CPC_OK;
  if (precision == CPC_FP64) {
    tri_gram_kernel<double, MODE_ROWS><<<grid, TPB, 0, s>>>(n, n_factors, N, U_items, a_axis,
        static_cast<const double*>(W_rho), b_axis, 1, nullptr, c_rho, P->R_N, rowpart, nullptr, tiles_per_cta);
    CPC_LAUNCH_CHECK("tri_gram_kernel(ROWS)");
  } else if (precision == CPC_SPLIT) {
    st = launch_rows32(P, n_factors, U_items, N, nullptr, c_rho, rowpart, groups, tiles_per_cta, s,
                       static_cast<const double*>(W_rho));
  } else if (tc_supported(P)) {
    // tensor cores over the R_rho R_N columns (m, q) as one-term factors
    // (layout in contract_bytes); with smooth terms, the dense columns
    // (m, dense term j) over the cells and the smooth ones from the moments
    const cpc_kernel Q = column_view(P);
    const int Nc = R_rho * P->R_N;
    const bool sm = cheb_scratch && coulomb_smooth(P);
    int n_dense = P->R_N;
    const int* dq = sm ? dense_terms(P, 0, &n_dense) : nullptr;
    const int n_sm = sm ? P->n_smooth[0] : 0;
    const int Nd = R_rho * n_dense, Ns = R_rho * n_sm;
    const cpc_kernel Qm = moment_view(P);
    unsigned char* w = reinterpret_cast<unsigned char*>(rowpart);
    double* cq = reinterpret_cast<double*>(w);
    w += align256(sizeof(double) * Nc);
    double* cqs = reinterpret_cast<double*>(w);
    if (sm) w += align256(sizeof(double) * Ns);
    const int tg_d = Nd > 0 ? (int)tc_rows_groups(&Q, Nd) : 0;
    const int tg_s = Ns > 0 ? (int)tc_rows_groups(&Qm, Ns) : 0;
    double* rp = reinterpret_cast<double*>(w);  // [tg_d + tg_s][n_factors]
    w += align256(sizeof(double) * (size_t)tc_rows_groups(&Q, Nc) * n_factors) +
         (sm ? align256(sizeof(double) * (size_t)tc_rows_groups(&Qm, Ns) * n_factors) : 0);
    void* tws = w;
    w += tc_rows_workspace(&Q, n_factors, Nc);
    const int* status = nullptr;
    const int* status2 = nullptr;
    if (Nd > 0) {
      expand_coef_kernel<<<(Nd + 255) / 256, 256, 0, s>>>(R_rho, n_dense, c_rho, cq);
      CPC_LAUNCH_CHECK("expand_coef_kernel");
      st = launch_rows_tc(&Q, n_factors, U_items, Nd, static_cast<const float*>(W_rho), cq, rp, tws, s, tiles_per_cta,
                          dq, n_dense, P->R_N);
      if (st) return st;
      status = tc_rows_status_ptr(&Q, n_factors, Nd, tws);
    }
    if (Ns > 0) {
      void* tws_s = w;
      w += tc_rows_workspace(&Qm, n_factors, Ns);
      double* A = reinterpret_cast<double*>(w);
      w += align256(sizeof(double) * 3 * size_t(n_factors) * kMomCells);
      float* B = reinterpret_cast<float*>(w);
      w += align256(sizeof(float) * 3 * size_t(Ns) * kMomCells);
      st = cheb_moment_rows(P, 3 * n_factors, U_items, w, A, kMomCells, s);
      if (st) return st;
      st = cheb_coef_rows(P, R_rho, cheb_scratch, B, kMomCells, s);
      if (st) return st;
      expand_coef_kernel<<<(Ns + 255) / 256, 256, 0, s>>>(R_rho, n_sm, c_rho, cqs);
      CPC_LAUNCH_CHECK("expand_coef_kernel");
      st = launch_rows_tc(&Qm, n_factors, A, Ns, B, cqs, rp + (size_t)tg_d * n_factors, tws_s, s, tiles_per_cta);
      if (st) return st;
      status2 = tc_rows_status_ptr(&Qm, n_factors, Ns, tws_s);
    }
    item_reduce_kernel<<<(n_items + 127) / 128, 128, 0, s>>>(n_items, off, c_items, rp, tg_d + tg_s, n_factors, scale,
                                                           J, status, status2);
    CPC_LAUNCH_CHECK("item_reduce_kernel");
    return CPC_OK;
  } else {
    st = launch_rows32(P, n_factors, U_items, N, static_cast<const float*>(W_rho), c_rho, rowpart, groups,
                       tiles_per_cta, s);
  }
  if (st) return st;
  item_reduce_kernel<<<(n_items + 127) / 128, 128, 0, s>>>(n_items, off, c_items, rowpart, groups, n_factors,
                                                         scale, J);
  CPC_LAUNCH_CHECK("item_reduce_kernel");
  return CPC_OK;
}

static int check_coulomb(const cpc_kernel* P, int n_items, const int* off, int n_factors, const double* U_items,
                         const double* c_items, int R_rho, const double* U_rho, const double* c_rho, void* W_rho,
                         double* J, int precision, int tiles_per_cta, void* ws, size_t ws_bytes, const char* who) {
  if (precision == CPC_FP64_TC)
    return fail(CPC_ERR_UNSUPPORTED, std::string(who) + ": CPC_FP64_TC is an E_H form; use CPC_FP64");
  int st = check_conv_args(P, R_rho, U_rho, W_rho, precision, ws, ws_bytes, who);
  if (st) return st;
  if (n_items <= 0 || !off || !U_items || !c_items || !c_rho || !J)
    return fail(CPC_ERR_INVALID, std::string(who) + ": bad item arguments");
  if (n_factors <= 0) return fail(CPC_ERR_INVALID, std::string(who) + ": no item factors");
  if (tiles_per_cta != 0 && (tiles_per_cta < 1 || tiles_per_cta > kTilesMax || (tiles_per_cta & (tiles_per_cta - 1))))
    return fail(CPC_ERR_INVALID, std::string(who) + ": tiles_per_cta must be 0 or a power of two in [1, 128]");
  if (ws_bytes < coulomb_matrix_workspace(P, n_items, n_factors, R_rho, precision))
    return fail(CPC_ERR_WORKSPACE, std::string(who) + ": workspace too small");
  return CPC_OK;
}
}  // namespace cpc

extern "C" size_t coulomb_matrix_workspace(const cpc_kernel* P, int n_items, int n_factors, int R_rho,
                                           int precision) {
  if (!P || n_items <= 0 || n_factors <= 0 || R_rho <= 0) return 0;
  return cp_convolve_workspace(P, R_rho, precision) + contract_bytes(P, n_factors, R_rho, precision);
}

extern "C" int coulomb_matrix(const cpc_kernel* P, int n_items, const int* off, int n_factors, const double* U_items,
                              const double* c_items, int R_rho, const double* U_rho, const double* c_rho,
                              void* W_rho, double* J, int precision, int tiles_per_cta, void* ws, size_t ws_bytes,
                              void* stream) {
  clear_error();
  int st = check_coulomb(P, n_items, off, n_factors, U_items, c_items, R_rho, U_rho, c_rho, W_rho, J, precision,
                         tiles_per_cta, ws, ws_bytes, "coulomb_matrix");
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = run_convolve(P, R_rho, U_rho, W_rho, precision, ws, s);
  if (st) return st;
  double* rowpart = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + cp_convolve_workspace(P, R_rho, precision));
  const void* scratch = static_cast<unsigned char*>(ws) + conv_spectra_bytes(P, R_rho, precision);
  return coulomb_contract(P, n_items, off, n_factors, U_items, c_items, R_rho, c_rho, W_rho, J, precision,
                          tiles_per_cta ? tiles_per_cta : kTilesDefault, rowpart, s, P->h * P->h * P->h, scratch);
}

extern "C" int coulomb_matrix_tune(const cpc_kernel* P, int n_items, const int* off, int n_factors,
                                   const double* U_items, const double* c_items, int R_rho, const double* U_rho,
                                   const double* c_rho, void* W_rho, double* J, int precision, void* ws,
                                   size_t ws_bytes, void* stream, int* best_tiles_per_cta, float* best_ms,
                                   float* times_ms) {
  clear_error();
  int st = check_coulomb(P, n_items, off, n_factors, U_items, c_items, R_rho, U_rho, c_rho, W_rho, J, precision, 0,
                         ws, ws_bytes, "coulomb_matrix_tune");
  if (st) return st;
  if (!best_tiles_per_cta) return fail(CPC_ERR_INVALID, "coulomb_matrix_tune: NULL best_tiles_per_cta");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = run_convolve(P, R_rho, U_rho, W_rho, precision, ws, s);
  if (st) return st;
  double* rowpart = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + cp_convolve_workspace(P, R_rho, precision));
  const void* scratch = static_cast<unsigned char*>(ws) + conv_spectra_bytes(P, R_rho, precision);
  // candidates: the tensor-core form (CPC_FP32, n a multiple of 128) rasters
  // its CTA pairs over groups of 1..32 item-row blocks; the CUDA-core forms
  // take 4..128 column tiles per work unit
  const bool tc = (precision == CPC_FP32 && tc_supported(P));
  const int lo = tc ? kRasterMin : kTilesMin, hi = tc ? kRasterMax : kTilesMax;
  // the events are released on every return path
  struct Events {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~Events() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ev;
  CPC_CUDA(cudaEventCreate(&ev.e[0]));
  CPC_CUDA(cudaEventCreate(&ev.e[1]));
  if (times_ms)
    for (int k = 0; k < 8; ++k) times_ms[k] = __builtin_nanf("");
  float best = -1.0f;
  int best_t = kTilesDefault;
  for (int t = lo; t <= hi; t *= 2) {
    // one untimed launch per candidate, then one timed
    st = coulomb_contract(P, n_items, off, n_factors, U_items, c_items, R_rho, c_rho, W_rho, J, precision, t, rowpart, s,
                          P->h * P->h * P->h, scratch);
    if (st) return st;
    CPC_CUDA(cudaEventRecord(ev.e[0], s));
    st = coulomb_contract(P, n_items, off, n_factors, U_items, c_items, R_rho, c_rho, W_rho, J, precision, t, rowpart, s,
                          P->h * P->h * P->h, scratch);
    if (st) return st;
    CPC_CUDA(cudaEventRecord(ev.e[1], s));
    CPC_CUDA(cudaEventSynchronize(ev.e[1]));
    float ms = 0.0f;
    CPC_CUDA(cudaEventElapsedTime(&ms, ev.e[0], ev.e[1]));
    if (times_ms) times_ms[ilog2(t)] = ms;
    if (best < 0.0f || ms < best) { best = ms; best_t = t; }
  }
  *best_tiles_per_cta = best_t;
  if (best_ms) *best_ms = best;
  // leave J computed with the chosen schedule
  return coulomb_contract(P, n_items, off, n_factors, U_items, c_items, R_rho, c_rho, W_rho, J, precision, best_t,
                          rowpart, s, P->h * P->h * P->h, scratch);
}

// ---- nuclear potential and its Galerkin matrix (Sec. 3.3) ---------------------
// V[t] = -sum_{r in item t} c_items[r] sum_a Z[a] sum_q prod_l <u_r^(l), F[l][a R_N + q]>,
// F the master kernel windowed onto each nucleus (launch_window): the Coulomb
// contraction with the nuclear factors in place of the V_H factors, the
// charges as their coefficients, and the scale -1 in place of h^3 (the
// Galerkin vectors already carry h^3).  In the tensor-core form the (a, q)
// columns are folded into one-term factors (10 nuclei x 51 terms: 4 tiles
// instead of one 10-column tile per term).
extern "C" size_t nuclear_matrix_workspace(const cpc_kernel* P, int n_items, int n_factors, int n_nuc,
                                           int precision) {
  if (!P || n_items <= 0 || n_factors <= 0 || n_nuc <= 0) return 0;
  return contract_bytes(P, n_factors, n_nuc, precision);
}

extern "C" int nuclear_matrix(const cpc_kernel* P, int n_items, const int* off, int n_factors, const double* U_items,
                              const double* c_items, int n_nuc, const int* nuc_edges, const double* Z, void* F,
                              double* V, int precision, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_MASTER) return fail(CPC_ERR_INVALID, "nuclear_matrix: needs a MASTER kernel");
  if (n_items <= 0 || n_factors <= 0 || !off || !U_items || !c_items || !nuc_edges || !Z || !F || !V)
    return fail(CPC_ERR_INVALID, "nuclear_matrix: bad arguments");
  if ((reinterpret_cast<uintptr_t>(U_items) & 15) || (reinterpret_cast<uintptr_t>(F) & 15))
    return fail(CPC_ERR_INVALID, "nuclear_matrix: U_items and F must be 16-byte aligned");
  if (precision != CPC_FP64 && precision != CPC_FP32 && precision != CPC_SPLIT)
    return fail(CPC_ERR_UNSUPPORTED, "nuclear_matrix: precision form not implemented");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(CPC_ERR_WORKSPACE, "nuclear_matrix: workspace NULL or not 256-byte aligned");
  if (ws_bytes < nuclear_matrix_workspace(P, n_items, n_factors, n_nuc, precision))
    return fail(CPC_ERR_WORKSPACE, "nuclear_matrix: workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = launch_window(P, n_nuc, nuc_edges, F, storage_precision(precision) == CPC_FP32, s);
  if (st) return st;
  return coulomb_contract(P, n_items, off, n_factors, U_items, c_items, n_nuc, Z, F, V, precision, kTilesDefault,
                          static_cast<double*>(ws), s, -1.0);
}

// ---- explicit spectra intermediates ------------------------------------------
extern "C" int cp_factor_spectra(const cpc_kernel* P, int R_f, const double* U, void* spec, int precision,
                                 void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_CONV || R_f <= 0 || !U || !spec)
    return fail(CPC_ERR_INVALID, "cp_factor_spectra: bad arguments");
  if (!known_precision(precision))
    return fail(CPC_ERR_UNSUPPORTED, "cp_factor_spectra: precision form not implemented");
  precision = storage_precision(precision);
  if ((reinterpret_cast<uintptr_t>(U) & 15) || (reinterpret_cast<uintptr_t>(spec) & 15))
    return fail(CPC_ERR_INVALID, "cp_factor_spectra: U and spec must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == CPC_FP64) return forward_spectra(P, 3 * R_f, U, static_cast<double2*>(spec), nullptr, s);
  return forward_spectra(P, 3 * R_f, U, nullptr, static_cast<float2*>(spec), s);
}

extern "C" int cp_convolve_from_spectra(const cpc_kernel* P, int R_f, const void* spec, void* W, int precision,
                                        void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_CONV || R_f <= 0 || !spec || !W)
    return fail(CPC_ERR_INVALID, "cp_convolve_from_spectra: bad arguments");
  if (!known_precision(precision))
    return fail(CPC_ERR_UNSUPPORTED, "cp_convolve_from_spectra: precision form not implemented");
  precision = storage_precision(precision);
  if ((reinterpret_cast<uintptr_t>(W) & 15) || (reinterpret_cast<uintptr_t>(spec) & 15))
    return fail(CPC_ERR_INVALID, "cp_convolve_from_spectra: spec and W must be 16-byte aligned");
  return convolve_from_spectra(P, 3 * R_f, spec, W, precision, static_cast<cudaStream_t>(stream));
}

extern "C" size_t cp_hartree_energy_from_spectra_workspace(const cpc_kernel* P, int R_f) {
  if (!P || R_f <= 0) return 0;
  return align256(sizeof(double) * eh32_partials(R_f, P->R_N));
}

extern "C" int cp_hartree_energy_from_spectra(const cpc_kernel* P, int R_f, const void* spec, const double* c,
                                              double* G, double* E_H, int precision, void* ws, size_t ws_bytes,
                                              void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_CONV || R_f <= 0 || !spec || !c || !E_H)
    return fail(CPC_ERR_INVALID, "cp_hartree_energy_from_spectra: bad arguments");
  if (precision != CPC_FP32)
    return fail(CPC_ERR_UNSUPPORTED, "cp_hartree_energy_from_spectra: only the float32 form contracts spectra");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) || ws_bytes < cp_hartree_energy_from_spectra_workspace(P, R_f))
    return fail(CPC_ERR_WORKSPACE, "cp_hartree_energy_from_spectra: workspace missing, misaligned or too small");
  return launch_eh_spectral(P, R_f, static_cast<const float2*>(spec), c, G, E_H, static_cast<double*>(ws),
                            static_cast<cudaStream_t>(stream));
}
