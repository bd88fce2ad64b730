// Self-test of the bounded device-side waits: the failure path of a wait that never completes,
// exercised without a fault or a hang.
#include "internal.cuh"
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

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_selftest_bounded_wait(hisq_ctx* ctx) {
  if (!ctx) return set_error(HISQ_EINVAL, "null context");
  int* d_flag = (int*)workspace(ctx, "selftest_flag", sizeof(int));
  if (!d_flag) return set_error(HISQ_ENOMEM, "self-test flag");
  HISQ_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), ctx->stream));
  k_selftest_wait<<<1, 32, 0, ctx->stream>>>(d_flag, 1u << 16);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  int flag = 0;
  HISQ_CUDA(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (flag == 1) return set_error(HISQ_ETIMEOUT, "self-test: the bounded wait gave up as intended");
  if (flag == 2) return set_error(HISQ_EINVAL, "self-test: a barrier nothing arrived at completed");
  return set_error(HISQ_ECUDA, "self-test kernel did not run");
}
