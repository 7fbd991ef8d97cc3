// float32 contractions on CUDA cores with a register-tiled GEMM core.
//
// gemm3_kernel computes, for row factors r and column factors s,
//   prod(r, s) = prod_{l=1..3} sum_kappa A_l[r][kappa] * B_l[s][kappa] * d(kappa)
// and reduces it like tri_gram_kernel (MODE 0: symmetric E_H partials over
// tiles with r <= s; MODE 1: per-row sums for Coulomb-matrix items).
// Two operand policies:
//   Spatial  : A = U (float64, rounded to float32 on load), B = V_H factors
//              (float32), d = 1, kappa = grid cell (Sec. 3.2 Eq. Factor_Mk_Conv).
//   Spectral : A = B = the factor spectra (float64-computed, float32-stored,
//              real view: kappa = 2f + {re, im}), d(kappa) = w_f p^_q[f] / (2n)
//              with w_0 = w_n = 1, else 2.  By Parseval on the length-2n circle
//              this is the same U^T (p_q * U) without reading the V_H factors.
// Each thread owns an 8 x 4 block of a 128 x 64 tile; K is staged through
// double-buffered shared memory 16 at a time; partial sums are float32 over
// chunks of 256 K values, then added into a float32 running total per axis
// (CPC_SPLIT: every 16-value block is folded into a compensated float32
// pair with FastTwoSum instead);
// the product over the three axes is kept in shared memory (one slot per
// thread and output) so the K loop keeps its registers for accumulators and
// operand fragments.  The spatial policy needs K (= n) even and U, W 16-byte
// aligned; the spectral policy K = 2(n+1).
#include <cuda_runtime.h>

#include <algorithm>

#include "cpc_internal.h"

namespace cpc {

namespace g32 {

constexpr int BM = 128, BN = 64, BK = 16, THREADS = 256;
constexpr int TMR = 8, TNC = 4;   // per-thread rows x cols
constexpr int CHUNK = 256;        // K values per float32 partial sum

struct Spatial {
  const double* A;   // [3][M][K]
  const float* B;    // [3][..][K], column s at (s * col_stride + col_off)
  long long a_axis, b_axis;
  int col_stride, col_off;
  int K;
  __device__ __forceinline__ float2 a2(int l, int r, int k) const {
    const double2 v = *reinterpret_cast<const double2*>(A + l * a_axis + (long long)r * K + k);
    return make_float2(float(v.x), float(v.y));
  }
  __device__ __forceinline__ float2 b2(int l, int s, int k) const {
    return *reinterpret_cast<const float2*>(B + l * b_axis + ((long long)s * col_stride + col_off) * K + k);
  }
};

// Spatial with float64 V_H factors rounded to float32 on load (CPC_SPLIT).
struct SpatialD {
  const double* A;
  const double* B;
  long long a_axis, b_axis;
  int col_stride, col_off;
  int K;
  __device__ __forceinline__ float2 a2(int l, int r, int k) const {
    const double2 v = *reinterpret_cast<const double2*>(A + l * a_axis + (long long)r * K + k);
    return make_float2(float(v.x), float(v.y));
  }
  __device__ __forceinline__ float2 b2(int l, int s, int k) const {
    const double2 v = *reinterpret_cast<const double2*>(B + l * b_axis + ((long long)s * col_stride + col_off) * K + k);
    return make_float2(float(v.x), float(v.y));
  }
};

struct Spectral {
  const float* S;    // [3][R_f][2(n+1)] real view of the spectra
  const float* d;    // [2(n+1)] weights of term q
  long long axis;
  int K;             // 2(n+1)
  __device__ __forceinline__ float2 a2(int l, int r, int k) const {
    return *reinterpret_cast<const float2*>(S + l * axis + (long long)r * K + k);
  }
  __device__ __forceinline__ float2 b2(int l, int s, int k) const {
    const float2 v = *reinterpret_cast<const float2*>(S + l * axis + (long long)s * K + k);
    const float2 w = __ldg(reinterpret_cast<const float2*>(d + k));
    return make_float2(v.x * w.x, v.y * w.y);
  }
};

// One axis: tot[8][4] = sum over K of A[r][k] B[s][k] for this thread's block.
// Loader: a warp covers 32 consecutive rows (columns) for one k range, so the
// transposed shared stores are conflict-free; loads are float2 where the
// operand allows (K is even and every k range starts on an even k).
template <class Op, bool COMP>
__device__ __forceinline__ void tile_axis(const Op& op, int l, int M, int N, int r0, int s0,
                                          float (&tot)[TMR][TNC], float* As, float* Bs) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int K = op.K;
  const int la_row = tid & (BM - 1), la_k = (tid >> 7) * 8;  // 128 rows x 2 halves of 8
  const int lb_col = tid & (BN - 1), lb_k = (tid >> 6) * 4;  // 64 cols x 4 quarters of 4
  float ra[8], rb[4];
  auto load = [&](int k0) {
    const int r = r0 + la_row;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      const int k = k0 + la_k + j;
      const bool ok = (r < M && k < K);  // k even, K even: k < K implies k + 1 < K
      const float2 v = ok ? op.a2(l, r, k) : make_float2(0.0f, 0.0f);
      ra[j] = v.x;
      ra[j + 1] = v.y;
    }
    const int s = s0 + lb_col;
#pragma unroll
    for (int j = 0; j < 4; j += 2) {
      const int k = k0 + lb_k + j;
      const bool ok = (s < N && k < K);
      const float2 v = ok ? op.b2(l, s, k) : make_float2(0.0f, 0.0f);
      rb[j] = v.x;
      rb[j + 1] = v.y;
    }
  };
  auto store = [&](int buf) {
    float* a = As + buf * BK * BM;
    float* b = Bs + buf * BK * BN;
#pragma unroll
    for (int j = 0; j < 8; ++j) a[(la_k + j) * BM + la_row] = ra[j];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[(lb_k + j) * BN + lb_col] = rb[j];
  };
#pragma unroll
  for (int i = 0; i < TMR; ++i)
#pragma unroll
    for (int j = 0; j < TNC; ++j) tot[i][j] = 0.0f;
  float acc[TMR][TNC], comp[TMR][TNC];
#pragma unroll
  for (int i = 0; i < TMR; ++i)
#pragma unroll
    for (int j = 0; j < TNC; ++j) { acc[i][j] = 0.0f; comp[i][j] = 0.0f; }
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const bool more = k0 + BK < K;
    if (more) load(k0 + BK);
    const float* a = As + buf * BK * BM + ty * TMR;
    const float* b = Bs + buf * BK * BN + tx * TNC;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(a + kk * BM);
      const float4 a1 = *reinterpret_cast<const float4*>(a + kk * BM + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(b + kk * BN);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b0.x, b0.y, b0.z, b0.w};
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TNC; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if constexpr (COMP) {
      // compensated: fold each 16-step block into (tot, comp) with FastTwoSum
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TNC; ++j) {
          const float s = tot[i][j] + acc[i][j];
          comp[i][j] += acc[i][j] - (s - tot[i][j]);
          tot[i][j] = s;
          acc[i][j] = 0.0f;
        }
    } else if (((k0 + BK) % CHUNK) == 0 || !more) {
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TNC; ++j) { tot[i][j] += acc[i][j]; acc[i][j] = 0.0f; }
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  if constexpr (COMP) {
#pragma unroll
    for (int i = 0; i < TMR; ++i)
#pragma unroll
      for (int j = 0; j < TNC; ++j) tot[i][j] += comp[i][j];
  }
  __syncthreads();  // smem reused by the next axis / tile
}

// dynamic shared memory: As[2][BK][BM], Bs[2][BK][BN], per-thread product slots [TMR*TNC][THREADS]
constexpr size_t kSmemBytes = sizeof(float) * (2 * BK * BM + 2 * BK * BN + TMR * TNC * THREADS);

template <class Op, int MODE, bool COMP = false>
__global__ void __launch_bounds__(THREADS, 2)
gemm3_kernel(Op op, int M, int N, const double* __restrict__ wr, const double* __restrict__ wcol, int wcol_div,
             double* __restrict__ partial, double* __restrict__ G, int n_rt, int tiles_per_cta,
             const float* __restrict__ dtab, long long d_stride, const int* __restrict__ qlist = nullptr,
             int R_N = 0) {
  extern __shared__ __align__(16) float smem[];
  float* As = smem;
  float* Bs = As + 2 * BK * BM;
  float* prod = Bs + 2 * BK * BN;  // prod[(i*TNC+j)*THREADS + tid]
  __shared__ double red[THREADS / 32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  auto P = [&](int i, int j) -> float& { return prod[(i * TNC + j) * THREADS + tid]; };
  if constexpr (MODE == 0) {
    // blockIdx.x enumerates (row tile, col tile) pairs; tiles entirely below
    // the diagonal (r > s everywhere) exit.  blockIdx.y is the kernel term q
    // (with qlist, the term qlist[blockIdx.y] of R_N).
    const int q = qlist ? __ldg(qlist + blockIdx.y) : int(blockIdx.y);
    const int n_terms = qlist ? R_N : int(gridDim.y);
    if constexpr (std::is_same<Op, Spectral>::value) op.d = dtab + (long long)q * d_stride;
    else op.col_off = q;
    const int n_ct = (N + BN - 1) / BN;
    const int rt = blockIdx.x / n_ct, ct = blockIdx.x % n_ct;
    const int r0 = rt * BM, s0 = ct * BN;
    double sum = 0.0;
    if (r0 <= s0 + BN - 1) {
      for (int l = 0; l < 3; ++l) {
        float tot[TMR][TNC];
        tile_axis<Op, COMP>(op, l, M, N, r0, s0, tot, As, Bs);
        if (G) {
          double* Gq = G + ((size_t)l * n_terms + q) * (size_t)M * M;
#pragma unroll
          for (int i = 0; i < TMR; ++i)
#pragma unroll
            for (int j = 0; j < TNC; ++j) {
              const int r = r0 + ty * TMR + i, s = s0 + tx * TNC + j;
              if (r < M && s < N && r <= s) {
                Gq[(size_t)r * M + s] = tot[i][j];
                Gq[(size_t)s * M + r] = tot[i][j];
              }
            }
        }
#pragma unroll
        for (int i = 0; i < TMR; ++i)
#pragma unroll
          for (int j = 0; j < TNC; ++j) P(i, j) = (l == 0) ? tot[i][j] : P(i, j) * tot[i][j];
      }
#pragma unroll
      for (int i = 0; i < TMR; ++i) {
        const int r = r0 + ty * TMR + i;
        if (r >= M) continue;
        double row = 0.0;
#pragma unroll
        for (int j = 0; j < TNC; ++j) {
          const int s = s0 + tx * TNC + j;
          if (s < N && r <= s) row += (r == s ? 1.0 : 2.0) * wcol[s] * double(P(i, j));
        }
        sum += wr[r] * row;
      }
    }
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((tid & 31) == 0) red[tid >> 5] = sum;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < THREADS / 32; ++w) s += red[w];
      partial[(size_t)q * gridDim.x + blockIdx.x] = s;
    }
  } else {
    // persistent over work units u = (row tile u % n_rt, column group u / n_rt)
    const int n_rtile = (M + BM - 1) / BM;
    const int n_ct = (N + BN - 1) / BN;
    const int n_groups = (n_ct + tiles_per_cta - 1) / tiles_per_cta;
    for (long long u = blockIdx.x; u < (long long)n_rtile * n_groups; u += gridDim.x) {
    const int rt = int(u % n_rtile), grp = int(u / n_rtile);
    const int r0 = rt * BM;
    double rowacc[TMR];
#pragma unroll
    for (int i = 0; i < TMR; ++i) rowacc[i] = 0.0;
    const int ct_end = min(n_ct, (grp + 1) * tiles_per_cta);
    for (int ct = grp * tiles_per_cta; ct < ct_end; ++ct) {
      const int s0 = ct * BN;
      for (int l = 0; l < 3; ++l) {
        float tot[TMR][TNC];
        tile_axis<Op, COMP>(op, l, M, N, r0, s0, tot, As, Bs);
#pragma unroll
        for (int i = 0; i < TMR; ++i)
#pragma unroll
          for (int j = 0; j < TNC; ++j) P(i, j) = (l == 0) ? tot[i][j] : P(i, j) * tot[i][j];
      }
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TNC; ++j) {
          const int s = s0 + tx * TNC + j;
          if (s < N) rowacc[i] += wcol[s / wcol_div] * double(P(i, j));
        }
    }
#pragma unroll
    for (int i = 0; i < TMR; ++i) {
      double v = rowacc[i];
      for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 16);
      const int r = r0 + ty * TMR + i;
      if (tx == 0 && r < M) partial[(size_t)grp * M + r] = v;
    }
    __syncthreads();  // prod slots are rewritten by the next unit
    }
  }
}

// d_q[kappa] = w_f p^_q[f] / (2n), kappa = 2f, 2f+1
__global__ void spectral_weights_kernel(int n, int R_N, const double* __restrict__ phat, float* __restrict__ d) {
  const int kappa = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  const int K = 2 * (n + 1);
  if (kappa >= K) return;
  const int f = kappa >> 1;
  const double w = (f == 0 || f == n) ? 1.0 : 2.0;
  d[(size_t)q * K + kappa] = float(w * phat[(size_t)q * (n + 1) + f] / (2.0 * n));
}

}  // namespace g32

size_t eh32_partials(int R_f, int R_N) {
  const int n_rt = (R_f + g32::BM - 1) / g32::BM, n_ct = (R_f + g32::BN - 1) / g32::BN;
  return size_t(n_rt) * n_ct * R_N;
}

int build_spectral_weights(const cpc_kernel* P, float* d, cudaStream_t s) {
  dim3 grid((2 * (P->n + 1) + 255) / 256, P->R_N);
  g32::spectral_weights_kernel<<<grid, 256, 0, s>>>(P->n, P->R_N, P->d_phat64, d);
  CPC_LAUNCH_CHECK("spectral_weights_kernel");
  return CPC_OK;
}

// E_H partial sums with float32 products; spectral (S32 != null), spatial on
// float32 factors (W) or spatial on float64 factors (W64, CPC_SPLIT).
int launch_eh32(const cpc_kernel* P, int R_f, const double* U, const float* W, const float* S32,
                const float* dtab, const double* c, double* G, double* partial, cudaStream_t s,
                const double* W64, const int* qlist, int n_q) {
  const int n_rt = (R_f + g32::BM - 1) / g32::BM, n_ct = (R_f + g32::BN - 1) / g32::BN;
  dim3 grid(n_rt * n_ct, P->R_N);
  if (W64) {
    // (a term list: the partial slots of the other terms are zeroed)
    if (qlist) {
      CPC_CUDA(cudaMemsetAsync(partial, 0, sizeof(double) * eh32_partials(R_f, P->R_N), s));
      if (n_q <= 0) return CPC_OK;
      grid.y = n_q;
    }
    g32::SpatialD op{U, W64, (long long)R_f * P->n, (long long)R_f * P->R_N * P->n, P->R_N, 0, P->n};
    CPC_CUDA(cudaFuncSetAttribute(g32::gemm3_kernel<g32::SpatialD, 0, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, int(g32::kSmemBytes)));
    g32::gemm3_kernel<g32::SpatialD, 0, true><<<grid, g32::THREADS, g32::kSmemBytes, s>>>(
        op, R_f, R_f, c, c, 1, partial, G, n_rt, 0, nullptr, 0, qlist, P->R_N);
  } else if (S32) {
    g32::Spectral op{S32, nullptr, (long long)R_f * 2 * (P->n + 1), 2 * (P->n + 1)};
    CPC_CUDA(cudaFuncSetAttribute(g32::gemm3_kernel<g32::Spectral, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(g32::kSmemBytes)));
    g32::gemm3_kernel<g32::Spectral, 0><<<grid, g32::THREADS, g32::kSmemBytes, s>>>(op, R_f, R_f, c, c, 1, partial, G, n_rt, 0,
                                                                       dtab, 2LL * (P->n + 1));
  } else {
    g32::Spatial op{U, W, (long long)R_f * P->n, (long long)R_f * P->R_N * P->n, P->R_N, 0, P->n};
    CPC_CUDA(cudaFuncSetAttribute(g32::gemm3_kernel<g32::Spatial, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(g32::kSmemBytes)));
    g32::gemm3_kernel<g32::Spatial, 0><<<grid, g32::THREADS, g32::kSmemBytes, s>>>(op, R_f, R_f, c, c, 1, partial, G, n_rt, 0,
                                                                      nullptr, 0);
  }
  CPC_LAUNCH_CHECK("gemm3_kernel(EH)");
  return CPC_OK;
}

// Coulomb rows with float32 products (spatial: item factors vs V_H factors,
// float32 factors W or float64 factors W64 for CPC_SPLIT).
int launch_rows32(const cpc_kernel* P, int n_factors, const double* U_items, int N, const float* W,
                  const double* c_rho, double* rowpart, int groups, int tiles_per_cta, cudaStream_t s,
                  const double* W64) {
  const long long units = (long long)((n_factors + g32::BM - 1) / g32::BM) * groups;
  const int grid = (int)std::min<long long>(units, 2LL * 152 * 2);
  if (W64) {
    g32::SpatialD op{U_items, W64, (long long)n_factors * P->n, (long long)N * P->n, 1, 0, P->n};
    CPC_CUDA(cudaFuncSetAttribute(g32::gemm3_kernel<g32::SpatialD, 1, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, int(g32::kSmemBytes)));
    g32::gemm3_kernel<g32::SpatialD, 1, true><<<grid, g32::THREADS, g32::kSmemBytes, s>>>(
        op, n_factors, N, nullptr, c_rho, P->R_N, rowpart, nullptr, 0, tiles_per_cta, nullptr, 0);
    CPC_LAUNCH_CHECK("gemm3_kernel(ROWS, split)");
    return CPC_OK;
  }
  g32::Spatial op{U_items, W, (long long)n_factors * P->n, (long long)N * P->n, 1, 0, P->n};
  CPC_CUDA(cudaFuncSetAttribute(g32::gemm3_kernel<g32::Spatial, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(g32::kSmemBytes)));
  g32::gemm3_kernel<g32::Spatial, 1><<<grid, g32::THREADS, g32::kSmemBytes, s>>>(op, n_factors, N, nullptr, c_rho, P->R_N,
                                                                    rowpart, nullptr, 0, tiles_per_cta, nullptr, 0);
  CPC_LAUNCH_CHECK("gemm3_kernel(ROWS)");
  return CPC_OK;
}

}  // namespace cpc
