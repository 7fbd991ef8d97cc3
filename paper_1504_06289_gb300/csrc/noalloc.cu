// cp_hartree_energy_noalloc: the Hartree energy for callers that cannot
// allocate device memory.
//
// Some hosts of this library own every byte of device memory themselves: an
// SCF program that reserves one fixed pool at start-up, a plug-in running
// inside another runtime's allocator, or a real-time loop that must not call
// cudaMalloc (it can synchronise the device and its latency is unbounded).
// Such callers can pass inputs and outputs but have no way to hand over a
// workspace.  This entry point takes its scratch from one file-scope device
// array of fixed size instead, so it allocates nothing at call time.
//
// The array is static device memory of the library's module: every GPU that
// loads the library holds kScratchBytes of it (per CUDA context) until the
// process exits.  All calls in a context share it and it keeps the previous
// call's contents; the kernels here overwrite every scratch byte they read
// (spectra and per-CTA partial sums; the tensor-core status word is cleared
// on every call), so nothing needs clearing by the caller.  Two calls whose
// work overlaps on the GPU (different streams, no ordering between them) race
// on the array.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "cpc_internal.h"

namespace cpc {

int check_conv_inputs(const cpc_kernel* P, int R_f, const void* U, const void* W, int precision,
                      const char* who);
int check_conv_args(const cpc_kernel* P, int R_f, const void* U, const void* W, int precision,
                    void* ws, size_t ws_bytes, const char* who);
int run_hartree_energy(const cpc_kernel* P, int R_f, const double* U, const double* c, void* W, double* G,
                       double* E_H, int precision, void* ws, cudaStream_t s);

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

int ctx_get_current_fn(CtxGetCurrentFn* out) {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
  });
  if (!fn) return fail(CPC_ERR_CUDA, "cp_hartree_energy_noalloc: cuCtxGetCurrent entry point unavailable");
  *out = fn;
  return CPC_OK;
}

// The array's device address per CUDA context.  A device address is only
// valid in the context it was looked up in (a caller's own non-primary
// context on a device gets its own copy of the module's device arrays, and
// cudaDeviceReset replaces the primary context), so the cache is keyed by the
// current context and refreshed by every call that is not under stream
// capture; under capture the address from an earlier call in the same context
// is used.
std::mutex g_scratch_mutex;
std::vector<std::pair<CUcontext, void*>> g_scratch_ptr;

int scratch_in_current_context(cudaStream_t s, void** out) {
  CtxGetCurrentFn get_ctx;
  int st = ctx_get_current_fn(&get_ctx);
  if (st) return st;
  // a runtime call on the stream first: it makes the primary context current
  // if the caller has none
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CPC_CUDA(cudaStreamIsCapturing(s, &cap));
  CUcontext ctx = nullptr;
  if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx)
    return fail(CPC_ERR_CUDA, "cp_hartree_energy_noalloc: no current CUDA context");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  auto it = g_scratch_ptr.begin();
  while (it != g_scratch_ptr.end() && it->first != ctx) ++it;
  if (cap != cudaStreamCaptureStatusNone) {
    if (it == g_scratch_ptr.end())
      return fail(CPC_ERR_INVALID,
                  "cp_hartree_energy_noalloc: the first call in a CUDA context must come before any stream capture");
    *out = it->second;
    return CPC_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cp_hartree_energy_noalloc: cudaGetSymbolAddress");
  if (it == g_scratch_ptr.end()) g_scratch_ptr.emplace_back(ctx, p);
  else it->second = p;
  *out = p;
  return CPC_OK;
}

}  // namespace
}  // namespace cpc

using namespace cpc;

extern "C" int cp_hartree_energy_noalloc(const cpc_kernel* P, int R_f, const double* U, const double* c,
                                         void* W, double* G, double* E_H, int precision, void* stream) {
  clear_error();
  const char* who = "cp_hartree_energy_noalloc";
  // invalid arguments are reported as such before the size limit is applied
  int st = check_conv_inputs(P, R_f, U, W, precision, who);
  if (st) return st;
  if (!c || !E_H) return fail(CPC_ERR_INVALID, "cp_hartree_energy_noalloc: NULL c or E_H");
  const size_t need = cp_hartree_energy_workspace(P, R_f, precision);
  if (need > kScratchBytes)
    return fail(CPC_ERR_UNSUPPORTED,
                "cp_hartree_energy_noalloc: this size needs " + std::to_string(need) +
                    " bytes of scratch but the fixed scratch array holds " + std::to_string(kScratchBytes) +
                    " (32 MiB); use cp_hartree_energy with a caller workspace");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  st = scratch_in_current_context(s, &ws);
  if (st) return st;
  st = check_conv_args(P, R_f, U, W, precision, ws, kScratchBytes, who);
  if (st) return st;
  return run_hartree_energy(P, R_f, U, c, W, G, E_H, precision, ws, s);
}
