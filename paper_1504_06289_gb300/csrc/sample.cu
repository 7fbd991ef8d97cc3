// Grid sampling of Gaussians (Sec. 3.1, Eq. disc_GTO), Hadamard products of
// factor pairs (Sec. 2.5, Eq. had) and the chain rule from factor gradients
// to Gaussian exponents and centres.
#include <cuda_runtime.h>

#include "cpc_internal.h"

namespace cpc {

__global__ void sample_kernel(int n, double b, double h, int R, const double* __restrict__ a,
                              const double* __restrict__ X, double* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y, l = blockIdx.z;
  if (i >= n) return;
  const double x = -b + (i + 0.5) * h;
  const double d = x - X[3 * k + l];
  const double e = a[k] * d * d;
  // exp(-e) is exactly 0 in float64 beyond e = 745.2 (below the smallest
  // subnormal): skip the call there (most cells of a narrow Gaussian)
  U[((size_t)l * R + k) * n + i] = (e > 746.0) ? 0.0 : exp(-e);
}

__global__ void hadamard_kernel(int n, int n_in, int n_pairs, const int* __restrict__ pa,
                                const int* __restrict__ pb, const double* __restrict__ F,
                                double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y, l = blockIdx.z;
  if (i >= n) return;
  const int ia = pa[r], ib = pb[r];
  double v = 0.0;
  if (ia >= 0 && ia < n_in && ib >= 0 && ib < n_in)
    v = F[((size_t)l * n_in + ia) * n + i] * F[((size_t)l * n_in + ib) * n + i];
  out[((size_t)l * n_pairs + r) * n + i] = v;
}

__global__ void pair_coef_kernel(int n_in, int n_pairs, const int* __restrict__ pa, const int* __restrict__ pb,
                                 const double* __restrict__ d, const double* __restrict__ scale,
                                 double* __restrict__ c_out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_pairs) return;
  const int ia = pa[r], ib = pb[r];
  double v = 0.0;
  if (ia >= 0 && ia < n_in && ib >= 0 && ib < n_in) v = d[ia] * d[ib] * (scale ? scale[r] : 1.0);
  c_out[r] = v;
}

// one block per Gaussian k: four reductions over (axis, cell)
__global__ void param_grad_kernel(int n, double b, double h, int R, const double* __restrict__ a,
                                  const double* __restrict__ X, const double* __restrict__ U,
                                  const double* __restrict__ dU, double* __restrict__ da,
                                  double* __restrict__ dX) {
  const int k = blockIdx.x;
  double sa = 0.0, sx[3] = {0.0, 0.0, 0.0};
  for (int l = 0; l < 3; ++l) {
    const double Xl = X[3 * k + l];
    const double* u = U + ((size_t)l * R + k) * n;
    const double* du = dU + ((size_t)l * R + k) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = (-b + (i + 0.5) * h) - Xl;
      const double g = du[i] * u[i];
      sa -= g * d * d;
      sx[l] += g * 2.0 * a[k] * d;
    }
  }
  __shared__ double red[4][32];
  double v[4] = {sa, sx[0], sx[1], sx[2]};
  for (int j = 0; j < 4; ++j) {
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v[j];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    if (threadIdx.x == 0) da[k] = t;
    else dX[3 * k + threadIdx.x - 1] = t;
  }
}

}  // namespace cpc

using namespace cpc;

extern "C" int cp_sample_gaussians(int n, double b, int R, const double* a, const double* X, double* U,
                                   void* stream) {
  clear_error();
  if (n <= 0 || R <= 0 || !(b > 0.0) || !a || !X || !U) return fail(CPC_ERR_INVALID, "cp_sample_gaussians: bad arguments");
  if (R > 65535) return fail(CPC_ERR_UNSUPPORTED, "cp_sample_gaussians: R > 65535");
  dim3 grid((n + 255) / 256, R, 3);
  sample_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, b, 2.0 * b / n, R, a, X, U);
  CPC_LAUNCH_CHECK("sample_kernel");
  return CPC_OK;
}

extern "C" int cp_hadamard_pairs(int n, int n_in, int n_pairs, const int* pa, const int* pb, const double* F,
                                 const double* d, const double* scale, double* out, double* c_out, void* stream) {
  clear_error();
  if (n <= 0 || n_in <= 0 || n_pairs <= 0 || !pa || !pb || !F || !out)
    return fail(CPC_ERR_INVALID, "cp_hadamard_pairs: bad arguments");
  if (n_pairs > 65535 * 64) return fail(CPC_ERR_UNSUPPORTED, "cp_hadamard_pairs: too many pairs");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int r0 = 0; r0 < n_pairs; r0 += 65535) {
    const int cnt = n_pairs - r0 < 65535 ? n_pairs - r0 : 65535;
    // out is [3][n_pairs][n]: launch per axis so the chunk keeps its axis stride
    for (int l = 0; l < 3; ++l) {
      dim3 grid((n + 255) / 256, cnt, 1);
      hadamard_kernel<<<grid, 256, 0, s>>>(n, n_in, cnt, pa + r0, pb + r0, F + (size_t)l * n_in * n,
                                          out + ((size_t)l * n_pairs + r0) * n);
      CPC_LAUNCH_CHECK("hadamard_kernel");
    }
  }
  if (c_out) {
    if (!d) return fail(CPC_ERR_INVALID, "cp_hadamard_pairs: c_out needs d");
    pair_coef_kernel<<<(n_pairs + 255) / 256, 256, 0, s>>>(n_in, n_pairs, pa, pb, d, scale, c_out);
    CPC_LAUNCH_CHECK("pair_coef_kernel");
  }
  return CPC_OK;
}

extern "C" int cp_gaussian_param_grad(int n, double b, int R, const double* a, const double* X, const double* U,
                                      const double* dU, double* da, double* dX, void* stream) {
  clear_error();
  if (n <= 0 || R <= 0 || !(b > 0.0) || !a || !X || !U || !dU || !da || !dX)
    return fail(CPC_ERR_INVALID, "cp_gaussian_param_grad: bad arguments");
  param_grad_kernel<<<R, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, b, 2.0 * b / n, R, a, X, U, dU, da, dX);
  CPC_LAUNCH_CHECK("param_grad_kernel");
  return CPC_OK;
}
