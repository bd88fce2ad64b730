// Self-test of the bounded device-side waits (an mbarrier completion wait of the tensor-core kernels and
// the grid-barrier wait of the fused CG update): the failure path of a wait that never completes,
// exercised without a fault or a hang.
#include "internal.cuh"
#include "solver_common.cuh"
#include "tc.cuh"

namespace hisq {

// One block waits on an mbarrier that nothing arrives at, with the same bounded wait the tensor-core
// kernels use for their completion barriers; when the wait gives up, the kernel records it and exits.
__global__ void k_selftest_wait(int* flag, uint32_t limit) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t addr = tc::smem_addr(&bar);
  if (threadIdx.x == 0) tc::mbar_init(addr, 1);
  __syncthreads();
  const bool completed = tc::mbar_wait(addr, 0, limit);  // phase 0 of a fresh barrier never completes
  if (threadIdx.x == 0) *flag = completed ? 2 : 1;
}

// One block waits at the fused CG update's grid barrier for a generation that nobody advances (the word
// is zero and no block arrives), with the update's own bounded wait; when it gives up, the kernel records it.
__global__ void k_selftest_grid_wait(int* flag, const unsigned* word, long limit) {
  const bool passed = grid_wait64(word, 0u, limit);
  if (threadIdx.x == 0) *flag = passed ? 2 : 1;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_selftest_bounded_wait(hisq_ctx* ctx) {
  if (!ctx) return set_error(HISQ_EINVAL, "null context");
  // flags [0] mbarrier wait, [1] grid-barrier wait; then the grid barrier's 64-bit word (8-byte aligned)
  int* d_flag = (int*)workspace(ctx, "selftest_flag", 2 * sizeof(int) + sizeof(unsigned long long));
  if (!d_flag) return set_error(HISQ_ENOMEM, "self-test flag");
  const unsigned* word = reinterpret_cast<const unsigned*>(d_flag + 2);
  HISQ_CUDA(cudaMemsetAsync(d_flag, 0, 2 * sizeof(int) + sizeof(unsigned long long), ctx->stream));
  k_selftest_wait<<<1, 32, 0, ctx->stream>>>(d_flag, 1u << 16);
  k_selftest_grid_wait<<<1, 32, 0, ctx->stream>>>(d_flag + 1, word, 1L << 16);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx, 2);
  int flag[2] = {0, 0};
  HISQ_CUDA(cudaMemcpyAsync(flag, d_flag, sizeof flag, cudaMemcpyDeviceToHost, ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (flag[0] == 1 && flag[1] == 1)
    return set_error(HISQ_ETIMEOUT, "self-test: both bounded waits gave up as intended");
  if (flag[0] == 2 || flag[1] == 2) return set_error(HISQ_EINVAL, "self-test: a wait nothing could end completed");
  return set_error(HISQ_ECUDA, "self-test kernels did not run");
}
