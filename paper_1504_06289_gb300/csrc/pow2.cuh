// Powers of two as floats (exact scale factors).
#pragma once

#include <cuda_runtime.h>

namespace cpc {

// 2^k as a float, k in [-126, 127] (a normal float)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

}  // namespace cpc
