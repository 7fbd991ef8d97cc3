// float32 E_H contraction with an asynchronous-copy pipeline.
//
// Same mathematics as gemm3_kernel's spatial MODE 0 (Sec. 3.2 Eq.
// Factor_Mk_Conv, Sec. 2.5 Eq. scal): prod(r, s) = prod_l sum_i U_l[r][i] W_l[s*R_N+q][i],
// reduced with c_r c_s over r <= s.  Both operands are float32 in global
// memory (U is rounded once into the workspace by round_factors_kernel) and
// stream into shared memory with cp.async through a 4-stage pipeline, so no
// registers hold staged tiles.  Tiles are row-major ([row][16 k]) with the
// 16-byte chunk index XOR-swizzled by (row >> 1) & 3; a thread owns rows
// ty*8 + i and columns tx + 16 j, so the column fragment loads touch every
// bank group exactly twice (the two-wavefront minimum for 256 bytes).
#include <cuda_runtime.h>

#include <cstdint>

#include "cpc_internal.h"

namespace cpc {
namespace g32a {

constexpr int BM = 128, BN = 64, BK = 16, THREADS = 256, STAGES = 4;
constexpr int TMR = 8, TNC = 4;
constexpr int CHUNK = 256;
constexpr size_t kStageFloats = size_t(BM + BN) * BK;
constexpr size_t kSmemBytes = sizeof(float) * (STAGES * kStageFloats + size_t(TMR) * TNC * THREADS);

__device__ __forceinline__ int swz(int row, int c) { return c ^ ((row >> 1) & 3); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = valid ? 16 : 0;  // zero-fill rows beyond the matrix
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// U (float64) -> float32, same layout
__global__ void round_factors_kernel(const double* __restrict__ U, float* __restrict__ U32, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    U32[i] = float(U[i]);
}

struct Args {
  const float* A;   // [3][M][K]
  const float* B;   // [3][N*R_N][K]; column s of term q at row s*R_N + q
  long long a_axis, b_axis;
  int M, N, K, R_N;
  const double* c;
  double* partial;
  double* G;
};

// load k-step t of axis l into stage slot
__device__ __forceinline__ void issue_stage(const Args& g, float* stage, int l, int q, int r0, int s0, int t) {
  const int tid = threadIdx.x;
  const int k0 = t * BK;
  float* As = stage;
  float* Bs = stage + BM * BK;
  // A: 128 rows x 4 chunks = 512 chunks, two per thread
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int id = tid + h * THREADS;
    const int row = id >> 2, c = id & 3;
    const int r = r0 + row;
    const bool ok = r < g.M;
    const float* src = g.A + l * g.a_axis + (long long)(ok ? r : 0) * g.K + k0 + c * 4;
    cp_async16(As + row * BK + swz(row, c) * 4, src, ok);
  }
  // B: 64 rows x 4 chunks = 256 chunks, one per thread
  {
    const int row = tid >> 2, c = tid & 3;
    const int s = s0 + row;
    const bool ok = s < g.N;
    const float* src = g.B + l * g.b_axis + ((long long)(ok ? s : 0) * g.R_N + q) * g.K + k0 + c * 4;
    cp_async16(Bs + row * BK + swz(row, c) * 4, src, ok);
  }
}

__device__ __forceinline__ void axis_sum(const Args& g, float* smem, int l, int q, int r0, int s0,
                                         float (&tot)[TMR][TNC]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int T = g.K / BK;  // K is a multiple of 16
  float acc[TMR][TNC];
#pragma unroll
  for (int i = 0; i < TMR; ++i)
#pragma unroll
    for (int j = 0; j < TNC; ++j) { acc[i][j] = 0.0f; tot[i][j] = 0.0f; }
#pragma unroll
  for (int t = 0; t < STAGES - 1; ++t) {
    if (t < T) issue_stage(g, smem + t * kStageFloats, l, q, r0, s0, t);
    cp_async_commit();
  }
  for (int t = 0; t < T; ++t) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    {
      const int tn = t + STAGES - 1;
      if (tn < T) issue_stage(g, smem + (tn % STAGES) * kStageFloats, l, q, r0, s0, tn);
      cp_async_commit();
    }
    const float* As = smem + (t % STAGES) * kStageFloats;
    const float* Bs = As + BM * BK;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float4 b[TNC];
#pragma unroll
      for (int j = 0; j < TNC; ++j) {
        const int row = tx + 16 * j;
        b[j] = *reinterpret_cast<const float4*>(Bs + row * BK + swz(row, c) * 4);
      }
#pragma unroll
      for (int i = 0; i < TMR; ++i) {
        const int row = ty * TMR + i;
        const float4 a = *reinterpret_cast<const float4*>(As + row * BK + swz(row, c) * 4);
#pragma unroll
        for (int j = 0; j < TNC; ++j) {
          acc[i][j] = fmaf(a.x, b[j].x, acc[i][j]);
          acc[i][j] = fmaf(a.y, b[j].y, acc[i][j]);
          acc[i][j] = fmaf(a.z, b[j].z, acc[i][j]);
          acc[i][j] = fmaf(a.w, b[j].w, acc[i][j]);
        }
      }
    }
    if (((t + 1) * BK) % CHUNK == 0 || t == T - 1) {
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TNC; ++j) { tot[i][j] += acc[i][j]; acc[i][j] = 0.0f; }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

__global__ void __launch_bounds__(THREADS, 2) gemm3a_kernel(Args g) {
  extern __shared__ __align__(16) float smem[];
  float* prod = smem + STAGES * kStageFloats;  // prod[(i*TNC+j)*THREADS + tid]
  __shared__ double red[THREADS / 32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int q = blockIdx.y;
  const int n_ct = (g.N + BN - 1) / BN;
  const int rt = blockIdx.x / n_ct, ct = blockIdx.x % n_ct;
  const int r0 = rt * BM, s0 = ct * BN;
  double sum = 0.0;
  if (r0 <= s0 + BN - 1) {
    for (int l = 0; l < 3; ++l) {
      float tot[TMR][TNC];
      axis_sum(g, smem, l, q, r0, s0, tot);
      if (g.G) {
        double* Gq = g.G + ((size_t)l * gridDim.y + q) * (size_t)g.M * g.M;
#pragma unroll
        for (int i = 0; i < TMR; ++i)
#pragma unroll
          for (int j = 0; j < TNC; ++j) {
            const int r = r0 + ty * TMR + i, s = s0 + tx + 16 * j;
            if (r < g.M && s < g.N && r <= s) {
              Gq[(size_t)r * g.M + s] = tot[i][j];
              Gq[(size_t)s * g.M + r] = tot[i][j];
            }
          }
      }
#pragma unroll
      for (int i = 0; i < TMR; ++i)
#pragma unroll
        for (int j = 0; j < TNC; ++j) {
          float& p = prod[(i * TNC + j) * THREADS + tid];
          p = (l == 0) ? tot[i][j] : p * tot[i][j];
        }
    }
#pragma unroll
    for (int i = 0; i < TMR; ++i) {
      const int r = r0 + ty * TMR + i;
      if (r >= g.M) continue;
      double row = 0.0;
#pragma unroll
      for (int j = 0; j < TNC; ++j) {
        const int s = s0 + tx + 16 * j;
        if (s < g.N && r <= s) row += (r == s ? 1.0 : 2.0) * g.c[s] * double(prod[(i * TNC + j) * THREADS + tid]);
      }
      sum += g.c[r] * row;
    }
  }
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if ((tid & 31) == 0) red[tid >> 5] = sum;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < THREADS / 32; ++w) s += red[w];
    g.partial[(size_t)q * gridDim.x + blockIdx.x] = s;
  }
}

}  // namespace g32a

size_t eh32a_partials(int R_f, int R_N) {
  const int n_rt = (R_f + g32a::BM - 1) / g32a::BM, n_ct = (R_f + g32a::BN - 1) / g32a::BN;
  return size_t(n_rt) * n_ct * R_N;
}

size_t eh32a_u32_bytes(const cpc_kernel* P, int R_f) { return align256(sizeof(float) * 3 * size_t(R_f) * P->n); }

// U32: workspace for the float32 copy of U (eh32a_u32_bytes); W: float32 V_H factors.
int launch_eh32a(const cpc_kernel* P, int R_f, const double* U, const float* W, const double* c, double* G,
                 double* partial, float* U32, cudaStream_t s) {
  const long long count = 3LL * R_f * P->n;
  g32a::round_factors_kernel<<<(unsigned)std::min<long long>((count + 255) / 256, 4096), 256, 0, s>>>(U, U32, count);
  CPC_LAUNCH_CHECK("round_factors_kernel");
  const int n_rt = (R_f + g32a::BM - 1) / g32a::BM, n_ct = (R_f + g32a::BN - 1) / g32a::BN;
  dim3 grid(n_rt * n_ct, P->R_N);
  g32a::Args g{U32, W, (long long)R_f * P->n, (long long)R_f * P->R_N * P->n, R_f, R_f, P->n, P->R_N, c, partial, G};
  CPC_CUDA(cudaFuncSetAttribute(g32a::gemm3a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(g32a::kSmemBytes)));
  g32a::gemm3a_kernel<<<grid, g32a::THREADS, g32a::kSmemBytes, s>>>(g);
  CPC_LAUNCH_CHECK("gemm3a_kernel");
  return CPC_OK;
}

}  // namespace cpc
