// Two-electron integrals by 1D density fitting and a truncated Cholesky
// factorisation of the TEI matrix (Sec. 3.2), float64 throughout.
//
// Basis: N_b s-type primitive Gaussians (rank 1 each, sampled factors
// U_prims[l][mu][i]); pairs P = (pa[P], pb[P]).  Per axis l the side matrix
// G^(l)[i, P] = U[l][pa[P]][i] U[l][pb[P]][i] (n x N_P) is never stored.
//
//   1. 1D density fitting (Eq. 1DDensFit): truncated Cholesky with diagonal
//      pivoting of A = G G^T (columns A[:, p] = G G[p, :]^T formed on the fly),
//      stopped when the largest remaining diagonal is <= tol_df max diag(A);
//      U = L L[I, :]^{-1} (n x R_l), V = G[I, :]^T (N_P x R_l).
//   2. M_k^(l) = U^(l)T (p_k * U^(l)) (Eq. Factor_Mk_Conv) by cp_hartree_energy
//      (its convolution matrices G), the factors padded to R_max columns.
//   3. B = h^3 sum_k (.)_l V^(l) M_k^(l) V^(l)T: its diagonal, and the column
//      of each pivot, B[:, j] = h^3 sum_k prod_l V^(l) (M_k^(l) V^(l)[j, :]^T),
//      drive the same truncated Cholesky, B ~ L L^T (stopped at tol_b).
//   4. J(D) = L (L^T d) for a density matrix D (tei_coulomb).
//
// The pivot loop stays on the device: each step is a pick kernel (argmax of
// the remaining diagonal, or a stop flag), a column kernel and an update
// kernel; a step after the stop does nothing, so no host synchronisation is
// needed and the ranks are read from device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "cpc_internal.h"

namespace cpc {
namespace tei {

constexpr int kMaxRankDF = 128;  // columns of U per axis
constexpr int kThreads = 256;
constexpr int kPickThreads = 1024;
constexpr int kPairChunk = 4096;  // pivot-row values staged per pass in the side-matrix column

struct CholState {
  double stop;  // tol x largest initial diagonal
  double dp;    // diagonal at the current pivot
  int done;     // the stop rule has fired
  int rank;     // columns of L
};

// d[i] = sum_P G[i, P]^2
__global__ void side_diag_kernel(int n, int n_pairs, const double* __restrict__ U, const int* __restrict__ pa,
                                 const int* __restrict__ pb, double* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int P = 0; P < n_pairs; ++P) {
    const double g = U[(size_t)pa[P] * n + i] * U[(size_t)pb[P] * n + i];
    s += g * g;
  }
  d[i] = s;
}

// state: stop = tol max(d), done = 0, rank = 0
__global__ void __launch_bounds__(kPickThreads) init_state_kernel(int N, const double* __restrict__ d, double tol,
                                                                  CholState* st) {
  __shared__ double red[kPickThreads / 32];
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += kPickThreads) m = fmax(m, d[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < kPickThreads / 32; ++w) mm = fmax(mm, red[w]);
    st->stop = tol * mm;
    st->dp = 0.0;
    st->done = 0;
    st->rank = 0;
  }
}

// pivot of step s: the largest remaining diagonal (smallest index on ties)
__global__ void __launch_bounds__(kPickThreads) pick_kernel(int N, const double* __restrict__ d, int s,
                                                            CholState* st, int* __restrict__ piv) {
  if (st->done) return;  // uniform
  __shared__ double bv[kPickThreads / 32];
  __shared__ int bi[kPickThreads / 32];
  double v = -1.0;
  int idx = 0x7fffffff;
  for (int i = threadIdx.x; i < N; i += kPickThreads)
    if (d[i] > v) { v = d[i]; idx = i; }
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (v2 > v || (v2 == v && i2 < idx)) { v = v2; idx = i2; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = v; bi[threadIdx.x >> 5] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kPickThreads / 32; ++w)
      if (bv[w] > v || (bv[w] == v && bi[w] < idx)) { v = bv[w]; idx = bi[w]; }
    if (!(v > st->stop)) {
      st->done = 1;
      st->rank = s;
    } else {
      piv[s] = idx;
      st->dp = v;
      st->rank = s + 1;
    }
  }
}

// c[i] = A[i, p] = sum_P G[i, P] G[p, P], p the pivot of step s; block of
// 32 points x 8 pair groups (pairs P = g mod 8), summed in a fixed order
constexpr int kRows = 32, kGroups = 8;
__global__ void __launch_bounds__(kRows * kGroups)
side_column_kernel(int n, int n_pairs, const double* __restrict__ U, const int* __restrict__ pa,
                   const int* __restrict__ pb, const CholState* st, const int* __restrict__ piv, int s,
                   double* __restrict__ c) {
  if (st->done) return;
  __shared__ double gp[kPairChunk];
  __shared__ double red[kGroups][kRows];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kRows + tx;
  const int p = piv[s];
  const int i = blockIdx.x * kRows + tx;
  double acc = 0.0;
  for (int P0 = 0; P0 < n_pairs; P0 += kPairChunk) {
    const int cnt = min(kPairChunk, n_pairs - P0);
    __syncthreads();
    for (int k = tid; k < cnt; k += kRows * kGroups)
      gp[k] = U[(size_t)pa[P0 + k] * n + p] * U[(size_t)pb[P0 + k] * n + p];
    __syncthreads();
    if (i < n)
      for (int k = ty; k < cnt; k += kGroups)
        acc += U[(size_t)pa[P0 + k] * n + i] * U[(size_t)pb[P0 + k] * n + i] * gp[k];
  }
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && i < n) {
    double t = 0.0;
    for (int g = 0; g < kGroups; ++g) t += red[g][tx];
    c[i] = t;
  }
}

// column s of L from the pivot column c: L[s][i] = (c[i] - sum_{t<s} L[t][i] L[t][p]) / sqrt(d_p),
// and the remaining diagonal d[i] -= L[s][i]^2; block of 32 rows x 8 groups of
// earlier columns (t = g mod 8), summed in a fixed order
__global__ void __launch_bounds__(kRows * kGroups)
update_kernel(int N, int s, size_t ld, double* __restrict__ L, const double* __restrict__ c, double* __restrict__ d,
              const CholState* st, const int* __restrict__ piv) {
  if (st->done) return;
  __shared__ double red[kGroups][kRows];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * kRows + tx;
  const int p = piv[s];
  double acc = 0.0;
  if (i < N)
    for (int t = ty; t < s; t += kGroups) acc += L[t * ld + i] * L[t * ld + p];
  red[ty][tx] = acc;
  __syncthreads();
  if (ty == 0 && i < N) {
    double v = c[i];
    for (int g = 0; g < kGroups; ++g) v -= red[g][tx];
    const double l = v / sqrt(st->dp);
    L[s * ld + i] = l;
    d[i] -= l * l;
  }
}

// U[u][i] = (L L[I, :]^{-1})[i][u] for u < rank (backward substitution over u,
// L[I, :] lower triangular in pivot order), 0 for rank <= u < R_max
__global__ void __launch_bounds__(kThreads)
fit_solve_kernel(int n, int R_max, const double* __restrict__ L, const int* __restrict__ piv, const CholState* st,
                 double* __restrict__ Uf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = st->rank;
  for (int u = R_max - 1; u >= r; --u) Uf[(size_t)u * n + i] = 0.0;
  for (int u = r - 1; u >= 0; --u) {
    double acc = L[(size_t)u * n + i];
    for (int t = u + 1; t < r; ++t) acc -= Uf[(size_t)t * n + i] * L[(size_t)u * n + piv[t]];
    Uf[(size_t)u * n + i] = acc / L[(size_t)u * n + piv[u]];
  }
}

// V[P][t] = G[piv[t], P] for t < rank, 0 beyond
__global__ void pivot_rows_kernel(int n, int n_pairs, int R_max, const double* __restrict__ U, const int* __restrict__ pa,
                                  const int* __restrict__ pb, const int* __restrict__ piv, const CholState* st,
                                  double* __restrict__ V) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)n_pairs * R_max) return;
  const int P = int(k / R_max), t = int(k % R_max);
  double v = 0.0;
  if (t < st->rank) {
    const int p = piv[t];
    v = U[(size_t)pa[P] * n + p] * U[(size_t)pb[P] * n + p];
  }
  V[k] = v;
}

// threads (k, i): 64 kernel terms (k = tx, tx + 64, ...) x 16 pairs per block;
// the sum over k is reduced in a fixed order
constexpr int kTermThreads = 64, kPairRows = 16;

__device__ __forceinline__ double reduce_terms(double acc, double (*red)[2], int tx, int ty) {
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tx & 31) == 0) red[ty][tx >> 5] = acc;
  __syncthreads();
  return red[ty][0] + red[ty][1];
}

// B[i][i] = h^3 sum_k prod_l V_l[i] M_l[k] V_l[i]^T
__global__ void __launch_bounds__(kTermThreads * kPairRows)
tei_diag_kernel(int n_pairs, int R_max, int R_N, const double* __restrict__ V, const double* __restrict__ M,
                const CholState* fit, double h3, double* __restrict__ d) {
  __shared__ double red[kPairRows][2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * kPairRows + ty;
  double acc = 0.0;
  if (i < n_pairs)
    for (int k = tx; k < R_N; k += kTermThreads) {
      double prod = 1.0;
      for (int l = 0; l < 3; ++l) {
        const int r = fit[l].rank;
        const double* v = V + ((size_t)l * n_pairs + i) * R_max;
        const double* Mk = M + ((size_t)l * R_N + k) * R_max * R_max;
        double q = 0.0;
        for (int a = 0; a < r; ++a) {
          double row = 0.0;
          for (int b2 = 0; b2 < r; ++b2) row += Mk[(size_t)a * R_max + b2] * v[b2];
          q += v[a] * row;
        }
        prod *= q;
      }
      acc += prod;
    }
  const double tot = reduce_terms(acc, red, tx, ty);
  if (tx == 0 && i < n_pairs) d[i] = h3 * tot;
}

// wT[l][a][k] = sum_b M_l[k][a][b] V_l[j][b], j the pivot of step s; block (k, l)
__global__ void tei_w_kernel(int n_pairs, int R_max, int R_N, const double* __restrict__ V,
                             const double* __restrict__ M, const CholState* fit, const CholState* st,
                             const int* __restrict__ piv, int s, double* __restrict__ wT) {
  if (st->done) return;
  const int k = blockIdx.x, l = blockIdx.y, a = threadIdx.x;
  if (a >= R_max) return;
  const int r = fit[l].rank;
  const int j = piv[s];
  const double* v = V + ((size_t)l * n_pairs + j) * R_max;
  const double* Mk = M + ((size_t)l * R_N + k) * R_max * R_max;
  double acc = 0.0;
  if (a < r)
    for (int b2 = 0; b2 < r; ++b2) acc += Mk[(size_t)a * R_max + b2] * v[b2];
  wT[((size_t)l * R_max + a) * R_N + k] = acc;
}

// c[i] = B[i][j] = h^3 sum_k prod_l V_l[i] . w[l][k]
__global__ void __launch_bounds__(kTermThreads * kPairRows)
tei_column_kernel(int n_pairs, int R_max, int R_N, const double* __restrict__ V, const double* __restrict__ wT,
                  const CholState* fit, const CholState* st, double h3, double* __restrict__ c) {
  if (st->done) return;
  __shared__ double red[kPairRows][2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * kPairRows + ty;
  double acc = 0.0;
  if (i < n_pairs)
    for (int k = tx; k < R_N; k += kTermThreads) {
      double prod = 1.0;
      for (int l = 0; l < 3; ++l) {
        const int r = fit[l].rank;
        const double* v = V + ((size_t)l * n_pairs + i) * R_max;
        const double* w = wT + (size_t)l * R_max * R_N + k;
        double q = 0.0;
        for (int a = 0; a < r; ++a) q += v[a] * w[(size_t)a * R_N];
        prod *= q;
      }
      acc += prod;
    }
  const double tot = reduce_terms(acc, red, tx, ty);
  if (tx == 0 && i < n_pairs) c[i] = h3 * tot;
}

__global__ void ranks_kernel(const CholState* fit, const CholState* st, int* __restrict__ ranks) {
  if (threadIdx.x == 0) {
    for (int l = 0; l < 3; ++l) ranks[l] = fit[l].rank;
    ranks[3] = st->rank;
  }
}

// ---- J(D) ------------------------------------------------------------------
// d[P] = (2 - delta) D[pa][pb]
__global__ void pair_density_kernel(int n_b, int n_pairs, const int* __restrict__ pa, const int* __restrict__ pb,
                                    const double* __restrict__ D, double* __restrict__ dv) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= n_pairs) return;
  const int a = pa[P], b = pb[P];
  dv[P] = (a == b ? 1.0 : 2.0) * D[(size_t)a * n_b + b];
}

// t[s] = sum_P L[s][P] d[P] for s < R_B; block s
__global__ void __launch_bounds__(kThreads) lt_d_kernel(int n_pairs, const double* __restrict__ L,
                                                        const double* __restrict__ dv, const int* __restrict__ ranks,
                                                        double* __restrict__ t) {
  __shared__ double red[kThreads / 32];
  const int s = blockIdx.x;
  if (s >= ranks[3]) {
    if (threadIdx.x == 0) t[s] = 0.0;
    return;
  }
  double acc = 0.0;
  for (int P = threadIdx.x; P < n_pairs; P += kThreads) acc += L[(size_t)s * n_pairs + P] * dv[P];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) tot += red[w];
    t[s] = tot;
  }
}

// J[P] = sum_{s < R_B} L[s][P] t[s]
__global__ void l_t_kernel(int n_pairs, const double* __restrict__ L, const double* __restrict__ t,
                           const int* __restrict__ ranks, double* __restrict__ J) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= n_pairs) return;
  const int r = ranks[3];
  double acc = 0.0;
  for (int s = 0; s < r; ++s) acc += L[(size_t)s * n_pairs + P] * t[s];
  J[P] = acc;
}

// ---- K(D) ------------------------------------------------------------------
// map[k][m] = the pair holding g_k g_m (either order), -1 if none
__global__ void pair_map_kernel(int n_b, int n_pairs, const int* __restrict__ pa, const int* __restrict__ pb,
                                int* __restrict__ map) {
  const int P = blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= n_pairs) return;
  const int a = pa[P], b = pb[P];
  if (a < 0 || a >= n_b || b < 0 || b >= n_b) return;  // outside the basis: no entry
  map[(size_t)a * n_b + b] = P;
  map[(size_t)b * n_b + a] = P;
}

// Z[s][k][nu] = sum_mu X_s[k][mu] D[mu][nu], X_s[k][mu] = L[s][map[k][mu]]; block (s, k)
__global__ void exchange_z_kernel(int n_b, int n_pairs, const double* __restrict__ L, const int* __restrict__ map,
                                  const int* __restrict__ ranks, const double* __restrict__ D,
                                  double* __restrict__ Z) {
  const int s = blockIdx.x, k = blockIdx.y, nu = threadIdx.x;
  if (s >= ranks[3] || nu >= n_b) return;
  const double* Ls = L + (size_t)s * n_pairs;
  double acc = 0.0;
  for (int mu = 0; mu < n_b; ++mu) {
    const int P = map[(size_t)k * n_b + mu];
    if (P >= 0) acc += Ls[P] * D[(size_t)mu * n_b + nu];
  }
  Z[((size_t)s * n_b + k) * n_b + nu] = acc;
}

// K[k][m] = sum_{s < R_B} sum_nu Z[s][k][nu] X_s[m][nu]
__global__ void exchange_k_kernel(int n_b, int n_pairs, const double* __restrict__ L, const int* __restrict__ map,
                                  const int* __restrict__ ranks, const double* __restrict__ Z,
                                  double* __restrict__ K) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
  if (m >= n_b) return;
  const int r = ranks[3];
  double acc = 0.0;
  for (int s = 0; s < r; ++s) {
    const double* Ls = L + (size_t)s * n_pairs;
    const double* z = Z + ((size_t)s * n_b + k) * n_b;
    for (int nu = 0; nu < n_b; ++nu) {
      const int P = map[(size_t)m * n_b + nu];
      if (P >= 0) acc += z[nu] * Ls[P];
    }
  }
  K[(size_t)k * n_b + m] = acc;
}

// workspace layout
struct Layout {
  size_t state, piv_fit, piv_b, dA, LA, c, Uf, V, M, W, hws, czero, E, dB, w, total;
};
inline Layout layout(const cpc_kernel* P, int n_pairs, int max_rank_b) {
  const size_t n = P->n, R = kMaxRankDF, RN = P->R_N;
  Layout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o += align256(bytes); return at; };
  L.state = take(4 * sizeof(CholState));
  L.piv_fit = take(3 * R * sizeof(int));
  L.piv_b = take(size_t(max_rank_b) * sizeof(int));
  L.dA = take(n * sizeof(double));
  L.LA = take(R * n * sizeof(double));
  L.c = take(std::max(n, size_t(n_pairs)) * sizeof(double));
  L.Uf = take(3 * R * n * sizeof(double));
  L.V = take(3 * size_t(n_pairs) * R * sizeof(double));
  L.M = take(3 * RN * R * R * sizeof(double));
  L.W = take(3 * R * RN * n * sizeof(double));
  L.hws = take(cp_hartree_energy_workspace(P, int(R), CPC_FP64));
  L.czero = take(R * sizeof(double));
  L.E = take(sizeof(double));
  L.dB = take(size_t(n_pairs) * sizeof(double));
  L.w = take(3 * RN * R * sizeof(double));
  L.total = o;
  return L;
}

}  // namespace tei
}  // namespace cpc

using namespace cpc;

extern "C" size_t tei_cholesky_workspace(const cpc_kernel* P, int n_pairs, int max_rank_b) {
  if (!P || n_pairs <= 0 || max_rank_b <= 0) return 0;
  return tei::layout(P, n_pairs, max_rank_b).total;
}

extern "C" int tei_cholesky(const cpc_kernel* P, int n_b, const double* U_prims, int n_pairs, const int* pa,
                            const int* pb, double tol_df, double tol_b, int max_rank_df, int max_rank_b, double* L,
                            int* ranks, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  if (!P || P->kind != CPC_KERNEL_CONV) return fail(CPC_ERR_INVALID, "tei_cholesky: needs a CONV kernel");
  if (n_b <= 0 || n_pairs <= 0 || !U_prims || !pa || !pb || !L || !ranks)
    return fail(CPC_ERR_INVALID, "tei_cholesky: bad arguments");
  if (!(tol_df >= 0.0) || !(tol_b >= 0.0)) return fail(CPC_ERR_INVALID, "tei_cholesky: tolerances must be >= 0");
  if (max_rank_df < 1 || max_rank_df > tei::kMaxRankDF)
    return fail(CPC_ERR_UNSUPPORTED, "tei_cholesky: max_rank_df must be in [1, 128]");
  if (max_rank_b < 1 || max_rank_b > n_pairs)
    return fail(CPC_ERR_INVALID, "tei_cholesky: max_rank_b must be in [1, n_pairs]");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(CPC_ERR_WORKSPACE, "tei_cholesky: workspace NULL or not 256-byte aligned");
  const tei::Layout Ly = tei::layout(P, n_pairs, max_rank_b);
  if (ws_bytes < Ly.total) return fail(CPC_ERR_WORKSPACE, "tei_cholesky: workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* w = static_cast<unsigned char*>(ws);
  auto at = [&](size_t off) { return w + off; };
  tei::CholState* st = reinterpret_cast<tei::CholState*>(at(Ly.state));  // [3] fits, [3] = TEI
  int* piv_fit = reinterpret_cast<int*>(at(Ly.piv_fit));
  int* piv_b = reinterpret_cast<int*>(at(Ly.piv_b));
  double* dA = reinterpret_cast<double*>(at(Ly.dA));
  double* LA = reinterpret_cast<double*>(at(Ly.LA));
  double* c = reinterpret_cast<double*>(at(Ly.c));
  double* Uf = reinterpret_cast<double*>(at(Ly.Uf));
  double* V = reinterpret_cast<double*>(at(Ly.V));
  double* M = reinterpret_cast<double*>(at(Ly.M));
  double* W = reinterpret_cast<double*>(at(Ly.W));
  double* czero = reinterpret_cast<double*>(at(Ly.czero));
  double* E = reinterpret_cast<double*>(at(Ly.E));
  double* dB = reinterpret_cast<double*>(at(Ly.dB));
  double* wv = reinterpret_cast<double*>(at(Ly.w));
  const int n = P->n, R = tei::kMaxRankDF, RN = P->R_N;
  const int T = tei::kThreads;
  // 1. density fitting per axis
  const int t_fit = timing_begin("tei_fit", s);
  for (int l = 0; l < 3; ++l) {
    const double* Ul = U_prims + (size_t)l * n_b * n;
    int* pv = piv_fit + l * R;
    tei::side_diag_kernel<<<(n + T - 1) / T, T, 0, s>>>(n, n_pairs, Ul, pa, pb, dA);
    tei::init_state_kernel<<<1, tei::kPickThreads, 0, s>>>(n, dA, tol_df, st + l);
    for (int step = 0; step < max_rank_df; ++step) {
      tei::pick_kernel<<<1, tei::kPickThreads, 0, s>>>(n, dA, step, st + l, pv);
      tei::side_column_kernel<<<(n + tei::kRows - 1) / tei::kRows, dim3(tei::kRows, tei::kGroups), 0, s>>>(
          n, n_pairs, Ul, pa, pb, st + l, pv, step, c);
      tei::update_kernel<<<(n + tei::kRows - 1) / tei::kRows, dim3(tei::kRows, tei::kGroups), 0, s>>>(
          n, step, size_t(n), LA, c, dA, st + l, pv);
    }
    tei::fit_solve_kernel<<<(n + T - 1) / T, T, 0, s>>>(n, R, LA, pv, st + l, Uf + (size_t)l * R * n);
    const long long nv = (long long)n_pairs * R;
    tei::pivot_rows_kernel<<<(unsigned)((nv + T - 1) / T), T, 0, s>>>(n, n_pairs, R, Ul, pa, pb, pv, st + l,
                                                                     V + (size_t)l * n_pairs * R);
    CPC_LAUNCH_CHECK("tei_cholesky: density fitting");
  }
  timing_end(t_fit, s);
  // 2. convolution matrices M_k^(l) = U^T (p_k * U)
  const int t_conv = timing_begin("tei_conv_matrices", s);
  CPC_CUDA(cudaMemsetAsync(czero, 0, R * sizeof(double), s));
  int st2 = cp_hartree_energy(P, R, Uf, czero, W, M, E, CPC_FP64, at(Ly.hws), cp_hartree_energy_workspace(P, R, CPC_FP64),
                              stream);
  timing_end(t_conv, s);
  if (st2) return st2;
  // 3. TEI diagonal and truncated Cholesky
  const int t_fac = timing_begin("tei_factor", s);
  const double h3 = P->h * P->h * P->h;
  tei::CholState* sb = st + 3;
  const dim3 tb(tei::kTermThreads, tei::kPairRows);
  const unsigned tg = (n_pairs + tei::kPairRows - 1) / tei::kPairRows;
  tei::tei_diag_kernel<<<tg, tb, 0, s>>>(n_pairs, R, RN, V, M, st, h3, dB);
  tei::init_state_kernel<<<1, tei::kPickThreads, 0, s>>>(n_pairs, dB, tol_b, sb);
  CPC_CUDA(cudaMemsetAsync(L, 0, sizeof(double) * (size_t)max_rank_b * n_pairs, s));
  for (int step = 0; step < max_rank_b; ++step) {
    tei::pick_kernel<<<1, tei::kPickThreads, 0, s>>>(n_pairs, dB, step, sb, piv_b);
    tei::tei_w_kernel<<<dim3(RN, 3), R, 0, s>>>(n_pairs, R, RN, V, M, st, sb, piv_b, step, wv);
    tei::tei_column_kernel<<<tg, tb, 0, s>>>(n_pairs, R, RN, V, wv, st, sb, h3, c);
    tei::update_kernel<<<(n_pairs + tei::kRows - 1) / tei::kRows, dim3(tei::kRows, tei::kGroups), 0, s>>>(
        n_pairs, step, size_t(n_pairs), L, c, dB, sb, piv_b);
  }
  tei::ranks_kernel<<<1, 32, 0, s>>>(st, sb, ranks);
  timing_end(t_fac, s);
  CPC_LAUNCH_CHECK("tei_cholesky: TEI factorisation");
  return CPC_OK;
}

extern "C" int tei_coulomb(int n_b, int n_pairs, const int* pa, const int* pb, int max_rank_b, const double* L,
                           const int* ranks, const double* D, double* J, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  if (n_b <= 0 || n_pairs <= 0 || max_rank_b <= 0 || !pa || !pb || !L || !ranks || !D || !J)
    return fail(CPC_ERR_INVALID, "tei_coulomb: bad arguments");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(CPC_ERR_WORKSPACE, "tei_coulomb: workspace NULL or not 256-byte aligned");
  if (ws_bytes < align256(sizeof(double) * n_pairs) + sizeof(double) * max_rank_b)
    return fail(CPC_ERR_WORKSPACE, "tei_coulomb: workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* dv = static_cast<double*>(ws);
  double* t = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + align256(sizeof(double) * n_pairs));
  const int T = tei::kThreads;
  tei::pair_density_kernel<<<(n_pairs + T - 1) / T, T, 0, s>>>(n_b, n_pairs, pa, pb, D, dv);
  tei::lt_d_kernel<<<max_rank_b, T, 0, s>>>(n_pairs, L, dv, ranks, t);
  tei::l_t_kernel<<<(n_pairs + T - 1) / T, T, 0, s>>>(n_pairs, L, t, ranks, J);
  CPC_LAUNCH_CHECK("tei_coulomb");
  return CPC_OK;
}

extern "C" size_t tei_exchange_workspace(int n_b, int max_rank_b) {
  if (n_b <= 0 || max_rank_b <= 0) return 0;
  return align256(sizeof(int) * (size_t)n_b * n_b) + sizeof(double) * (size_t)max_rank_b * n_b * n_b;
}

extern "C" int tei_exchange(int n_b, int n_pairs, const int* pa, const int* pb, int max_rank_b, const double* L,
                            const int* ranks, const double* D, double* K, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  if (n_b <= 0 || n_b > 1024 || n_pairs <= 0 || max_rank_b <= 0 || !pa || !pb || !L || !ranks || !D || !K)
    return fail(CPC_ERR_INVALID, "tei_exchange: bad arguments");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(CPC_ERR_WORKSPACE, "tei_exchange: workspace NULL or not 256-byte aligned");
  if (ws_bytes < tei_exchange_workspace(n_b, max_rank_b))
    return fail(CPC_ERR_WORKSPACE, "tei_exchange: workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* map = static_cast<int*>(ws);
  double* Z = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + align256(sizeof(int) * (size_t)n_b * n_b));
  CPC_CUDA(cudaMemsetAsync(map, 0xff, sizeof(int) * (size_t)n_b * n_b, s));  // -1
  const int T = tei::kThreads;
  tei::pair_map_kernel<<<(n_pairs + T - 1) / T, T, 0, s>>>(n_b, n_pairs, pa, pb, map);
  tei::exchange_z_kernel<<<dim3(max_rank_b, n_b), ((n_b + 31) / 32) * 32, 0, s>>>(n_b, n_pairs, L, map, ranks, D, Z);
  tei::exchange_k_kernel<<<dim3((n_b + 127) / 128, n_b), 128, 0, s>>>(n_b, n_pairs, L, map, ranks, Z, K);
  CPC_LAUNCH_CHECK("tei_exchange");
  return CPC_OK;
}
