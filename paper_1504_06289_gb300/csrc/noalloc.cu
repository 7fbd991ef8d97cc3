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
// loads the library holds kScratchBytes of it until the process exits.  All
// calls on a device share it and it keeps the previous call's contents; the
// kernels here overwrite every scratch byte they read (spectra and per-CTA
// partial sums), so nothing needs clearing.  Two calls whose work overlaps on
// the GPU (different streams, no ordering between them) race on the array.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "cpc_internal.h"

namespace cpc {

int check_conv_args(const cpc_kernel* P, int R_f, const void* U, const void* W, int precision,
                    void* ws, size_t ws_bytes, const char* who);
int run_hartree_energy(const cpc_kernel* P, int R_f, const double* U, const double* c, void* W, double* G,
                       double* E_H, int precision, void* ws, cudaStream_t s);

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int scratch_on_current_device(void** out) {
  int dev = 0;
  CPC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(CPC_ERR_UNSUPPORTED, "cp_hartree_energy_noalloc: device index beyond 63");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cp_hartree_energy_noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CPC_OK;
}

}  // namespace
}  // namespace cpc

using namespace cpc;

extern "C" int cp_hartree_energy_noalloc(const cpc_kernel* P, int R_f, const double* U, const double* c,
                                         void* W, double* G, double* E_H, int precision, void* stream) {
  clear_error();
  if (!P || R_f <= 0) return fail(CPC_ERR_INVALID, "cp_hartree_energy_noalloc: NULL kernel or R_f <= 0");
  if (!c || !E_H) return fail(CPC_ERR_INVALID, "cp_hartree_energy_noalloc: NULL c or E_H");
  const size_t need = cp_hartree_energy_workspace(P, R_f, precision);
  if (need > kScratchBytes)
    return fail(CPC_ERR_UNSUPPORTED,
                "cp_hartree_energy_noalloc: this size needs " + std::to_string(need) +
                    " bytes of scratch but the fixed scratch array holds " + std::to_string(kScratchBytes) +
                    " (32 MiB); use cp_hartree_energy with a caller workspace");
  void* ws = nullptr;
  int st = scratch_on_current_device(&ws);
  if (st) return st;
  st = check_conv_args(P, R_f, U, W, precision, ws, kScratchBytes, "cp_hartree_energy_noalloc");
  if (st) return st;
  return run_hartree_energy(P, R_f, U, c, W, G, E_H, precision, ws, static_cast<cudaStream_t>(stream));
}
