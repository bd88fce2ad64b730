// Sums of per-block partial results by one warp or by a whole block, in a fixed order: shared by the
// multi-RHS Dslash epilogues and the CG updates.
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

// Sum of partials[0..n) by a whole block (blockDim.x a multiple of 32), in a fixed order for a given n and
// block size; every thread gets the total. Up to 4 blockDim.x partials every thread's loads are in flight
// at once (one L2 round trip); beyond that warp 0 takes the loop above. red: blockDim.x / 32 doubles of
// shared memory, free again on return.
__device__ __forceinline__ double block_sum_partials(const double* partials, int n, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5, nb = blockDim.x;
  const bool wide = n <= 4 * nb;
  if (wide) {
    double v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = tid + k * nb < n ? __ldcg(partials + tid + k * nb) : 0.0;
    double t = (v[0] + v[1]) + (v[2] + v[3]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) red[warp] = t;
  } else if (warp == 0) {
    const double t = warp_sum_partials(partials, n);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  double s = red[0];
  if (wide)
    for (int w = 1; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

}  // namespace hisq
