// Solver state and BLAS-1 kernels shared by CG, mixed-precision CG and multi-shift CG.
//
// All iteration scalars (alpha, beta, residual norms, convergence flags) live in device
// memory, so a block of iterations runs without host round trips and can be captured in
// a CUDA graph. Reductions are FP64: per-block partial sums in a fixed order, combined
// by the last block to finish (deterministic for a fixed launch shape).
#pragma once
#include "internal.cuh"

namespace hisq {

constexpr int MAXR = 64;

struct SolverState {
  double rr[MAXR];       // iterated residual norm^2, in inner units
  double rr_new[MAXR];
  double pAp[MAXR];
  double bb[MAXR];       // ||b||^2
  double tol2[MAXR];     // (rel_tol * ||b||)^2, target for the true residual squared
  double scale[MAXR];    // true residual = scale * inner residual (mixed precision)
  double rr_true[MAXR];  // last FP64 true residual squared
  int rhs_done[MAXR];    // 1: inner-satisfied or verified; frozen (alpha = 0)
  int rhs_conv[MAXR];    // 1: true residual verified below tolerance
  int done;              // the current cycle of iterations is over
  int iter;              // iterations so far
  int cycle_iter;        // iterations in the current cycle
  int cycle_limit;       // cycle length (reliable period, or poll interval)
  int breakdown;
  int nonfinite;
  int nrhs;
  int pad;
};

// Reduce NQ per-rhs quantities over a 2D grid (x: sites, y: rhs) into partials[q][rhs][gx];
// returns true in the last block, whose thread 0 then finds totals in out[q][rhs].
template <int NQ>
__device__ __forceinline__ bool grid_reduce(double (&v)[NQ], double* partials, size_t pstride, unsigned* counter,
                                            double (&out)[NQ][MAXR], int nrhs) {
  __shared__ double red[32];
  const int gx = gridDim.x;
  const int r = blockIdx.y;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = block_sum_dyn(v[q], red);
    if (threadIdx.x == 0) partials[((size_t)q * MAXR + r) * pstride + blockIdx.x] = s;
  }
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  if (threadIdx.x == 0) *counter = 0u;
  for (int q = 0; q < NQ; ++q)
    for (int rr = 0; rr < nrhs; ++rr) {
      double s = sum_partials_dyn(partials + ((size_t)q * MAXR + rr) * pstride, gx, red);
      if (threadIdx.x == 0) out[q][rr] = s;
    }
  return true;
}

// Reduce one quantity per grid row (y = rhs) over the row's x-blocks: the last block of a row to finish
// sums that row's partials in block order, so the rows' tails overlap instead of queueing behind one
// block. row_counters[gridDim.y] start at zero and are reset by each row's last block. Returns true
// in every thread of that block; thread 0 then holds the row total in *total.
__device__ __forceinline__ bool row_reduce(double v, double* partials, size_t pstride, unsigned* row_counters,
                                           double* total) {
  __shared__ double red[32];
  __shared__ bool is_last;
  const int r = blockIdx.y;
  const double s = block_sum_dyn(v, red);
  if (threadIdx.x == 0) partials[(size_t)r * pstride + blockIdx.x] = s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(&row_counters[r], 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  if (threadIdx.x == 0) row_counters[r] = 0u;
  const double t = sum_partials_dyn(partials + (size_t)r * pstride, gridDim.x, red);
  if (threadIdx.x == 0) *total = t;
  return true;
}

template <typename S>
struct SAcc {
  using T = typename Real<S>::acc;
};

}  // namespace hisq
