// Warp-level sum of per-block partial results, shared by the multi-RHS Dslash and the CG updates.
#pragma once
#include <cuda_runtime.h>

namespace hisq {

// Sum of partials[0..n) by the 32 lanes of one warp, in a fixed order: eight independent accumulators
// per lane keep eight L2 loads in flight, then a fixed shuffle tree; every lane gets the total.
__device__ __forceinline__ double warp_sum_partials(const double* partials, int n) {
  const int lane = threadIdx.x & 31;
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int i = lane;
  for (; i + 7 * 32 < n; i += 8 * 32) {
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += __ldcg(partials + i + k * 32);
  }
  for (; i < n; i += 32) s[0] += __ldcg(partials + i);
  double t = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

}  // namespace hisq
