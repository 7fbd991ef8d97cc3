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
#include <cuda_runtime.h>

#include "cpc_internal.h"

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
  return launch_subgrid<float>(n, P->R_N, n_sub, S, sub, inv_h3, V, s);
}
