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
  double beta[MAXR];     // this iteration's beta = rr_new / rr (fused update: formed at its grid barrier)
  int rhs_done[MAXR];    // 1: inner-satisfied or verified; frozen (alpha = 0)
  int rhs_conv[MAXR];    // 1: true residual verified below tolerance
  int done;              // the current cycle of iterations is over
  int iter;              // iterations so far
  int cycle_iter;        // iterations in the current cycle
  int cycle_limit;       // cycle length (reliable period, or poll interval)
  int breakdown;
  int nonfinite;
  int nrhs;
  int timeout;           // a bounded grid-barrier wait of the fused update ran out
  // Lanczos coefficients of rhs 0 (CG's alpha and beta per iteration; alpha = 0 marks a restart of
  // the search direction), for the estimate of A's extreme eigenvalues: [2][lanczos_cap]
  double* lanczos;
  int lanczos_n;
  int lanczos_cap;
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

// ------------------------------------------------------------------ grid barrier (one-wave launches)
// The fused CG update runs as a cooperative launch (every block resident at once) and meets once per
// launch at a grid barrier: bar[0] counts arrivals, bar[1] is a generation number that the last block
// to arrive advances after its work. Waiting is bounded: after GRID_WAIT_POLLS polls the block gives up,
// the caller sets the solver's timeout flag and returns, so a barrier can never hang the GPU.
constexpr long GRID_WAIT_POLLS = 1L << 22;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Arrive at the barrier (every thread of every block). Returns true in every thread of the last block
// to arrive; *gen gets the generation this block must see advance before it may go on.
__device__ __forceinline__ bool grid_arrive(unsigned* bar, unsigned* gen) {
  __shared__ unsigned s_gen;
  __shared__ int s_last;
  __threadfence();  // this thread's writes (partials) become visible to the last block
  __syncthreads();
  const bool t0 = threadIdx.x == 0 && threadIdx.y == 0;
  if (t0) {
    s_gen = ld_acquire_gpu(bar + 1);
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    s_last = atomicAdd(bar, 1u) == nb - 1 ? 1 : 0;
  }
  __syncthreads();
  *gen = s_gen;
  return s_last != 0;
}

// The last block, after its work: reset the count and advance the generation (release).
__device__ __forceinline__ void grid_release(unsigned* bar) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    bar[0] = 0u;
    __threadfence();
    atomicAdd(bar + 1, 1u);
  }
  __syncthreads();
}

// The other blocks: wait (bounded) until the generation has advanced past gen. False on timeout.
__device__ __forceinline__ bool grid_wait(const unsigned* bar, unsigned gen) {
  __shared__ int s_ok;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int ok = 0;
    for (long it = 0; it < GRID_WAIT_POLLS; ++it) {
      if (ld_acquire_gpu(bar + 1) != gen) {
        ok = 1;
        break;
      }
      __nanosleep(64);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The same word read as one 64-bit value: bar[0] (arrivals) in the low half, bar[1] (generation) in the
// high half. With it the last block releases the others in the atomic right after its arrival, and the
// blocks then do their own post-barrier work in parallel (the fused CG update forms its sums that way).
__device__ __forceinline__ unsigned long long ld_acquire_gpu64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Arrive (every thread of every block, after the block's partial results are written) and, in the last
// block to arrive, release at once: one atomic adds 2^32 - nblocks (generation + 1, arrivals back to 0).
// *gen gets the generation to see advance; *last tells the block whether it arrived last.
__device__ __forceinline__ void grid_arrive_release(unsigned* bar, unsigned* gen, bool* last) {
  __shared__ unsigned s_gen;
  __shared__ int s_last;
  unsigned long long* w = reinterpret_cast<unsigned long long*>(bar);
  __threadfence();  // this block's partials become visible before its arrival
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned long long old = atomicAdd(w, 1ull);
    s_gen = (unsigned)(old >> 32);
    s_last = (unsigned)(old & 0xffffffffull) == nb - 1 ? 1 : 0;
    if (s_last) atomicAdd(w, (1ull << 32) - nb);
  }
  __syncthreads();
  *gen = s_gen;
  *last = s_last != 0;
}

// Wait (bounded) until the generation in the high half has advanced past gen (acquire: every block's
// partials are then visible). False on timeout.
__device__ __forceinline__ bool grid_wait64(const unsigned* bar, unsigned gen, long limit = GRID_WAIT_POLLS) {
  __shared__ int s_ok;
  const unsigned long long* w = reinterpret_cast<const unsigned long long*>(bar);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int ok = 0;
    for (long it = 0; it < limit; ++it) {
      if ((unsigned)(ld_acquire_gpu64(w) >> 32) != gen) {
        ok = 1;
        break;
      }
      __nanosleep(32);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename S>
struct SAcc {
  using T = typename Real<S>::acc;
};

}  // namespace hisq
