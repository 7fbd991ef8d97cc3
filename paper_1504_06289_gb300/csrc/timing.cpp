// Optional CUDA-event timing of the library's main kernels.  While enabled,
// each launch of a timed kernel is bracketed by two events recorded on the
// stream it is launched on; cpc_kernel_timing_read synchronises them and
// returns the summed device time per kernel name.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "cpc_internal.h"

namespace cpc {
namespace {

struct Slot {
  const char* name;
  cudaEvent_t a, b;
};

constexpr int kSlots = 8192;
std::mutex g_mu;
bool g_on = false;
std::vector<Slot> g_slots;  // events created when timing is first enabled
int g_used = 0;

}  // namespace

bool timing_on() { return g_on; }

int timing_begin(const char* name, cudaStream_t s) {
  if (!g_on) return -1;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on || g_used >= kSlots) return -1;
  const int i = g_used++;
  g_slots[i].name = name;
  if (cudaEventRecord(g_slots[i].a, s) != cudaSuccess) return -1;
  return i;
}

void timing_end(int slot, cudaStream_t s) {
  if (slot < 0) return;
  cudaEventRecord(g_slots[slot].b, s);
}

}  // namespace cpc

extern "C" int cpc_kernel_timing(int enable) {
  using namespace cpc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (enable) {
    if (g_slots.empty()) {
      g_slots.resize(kSlots);
      for (auto& sl : g_slots) {
        if (cudaEventCreate(&sl.a) != cudaSuccess || cudaEventCreate(&sl.b) != cudaSuccess) {
          g_slots.clear();
          return fail(CPC_ERR_CUDA, "cpc_kernel_timing: cudaEventCreate failed");
        }
      }
    }
    g_used = 0;
  }
  g_on = enable != 0;
  return CPC_OK;
}

extern "C" int cpc_kernel_timing_read(const char* kernel, double* total_ms, int* launches) {
  using namespace cpc;
  if (!kernel || !total_ms || !launches) return fail(CPC_ERR_INVALID, "cpc_kernel_timing_read: null argument");
  std::lock_guard<std::mutex> lk(g_mu);
  double tot = 0.0;
  int cnt = 0;
  for (int i = 0; i < g_used; ++i) {
    if (std::strcmp(g_slots[i].name, kernel) != 0) continue;
    if (cudaEventSynchronize(g_slots[i].b) != cudaSuccess) return fail(CPC_ERR_CUDA, "cpc_kernel_timing_read");
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, g_slots[i].a, g_slots[i].b) != cudaSuccess)
      return fail(CPC_ERR_CUDA, "cpc_kernel_timing_read: elapsed time");
    tot += ms;
    ++cnt;
  }
  *total_ms = tot;
  *launches = cnt;
  return CPC_OK;
}
