// Launch autotuner: the first launch of a kernel under a given key (kernel, precisions,
// rhs group, epilogue; the context fixes the lattice) times each candidate form and block size
// with CUDA events on the context's stream and keeps the fastest. Only idempotent
// kernels are tuned this way (the Dslash family: out = f(in) with no read of out).
// Inside a stream capture nothing is timed: an untuned key falls back to 256 threads.
#pragma once
#include <stdio.h>

#include <functional>

#include "internal.cuh"

namespace hisq {

// Grid cap for grid-stride kernels: two waves of a fully occupied GPU.
inline int max_grid_blocks(const hisq_ctx* ctx, int block) { return ctx->num_sms * (2048 / block) * 2; }
// Room per rhs in reduction-partials buffers (covers the smallest tuned block, 64).
inline size_t partial_stride(const hisq_ctx* ctx) { return (size_t)ctx->num_sms * 64; }

// One candidate kernel form for the tuner: its function (for the block-size limit) and a launcher
// taking the block size.
struct TuneVariant {
  const void* func;
  std::function<cudaError_t(int)> run;
};

// Times every (variant, block size) pair once per key and caches the fastest as
// variant * 10000 + block. With one variant this is a plain block-size tuner.
inline int tuned_variant(hisq_ctx* ctx, const char* key, const TuneVariant* v, int nv, int* vi_out, int* block_out) {
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end() && it->second > 0) {
    *vi_out = it->second / 10000;
    *block_out = it->second % 10000;
    return HISQ_OK;
  }
  if (it != ctx->tune.end()) {
    // a choice loaded from a report (stored negated until checked) is kept only if it names an
    // existing form and a block size that form can launch; otherwise the key is tuned again
    const int vi = -it->second / 10000, b = -it->second % 10000;
    cudaFuncAttributes fa;
    if (vi < nv && b >= 32 && b % 32 == 0 &&
        cudaFuncGetAttributes(&fa, v[vi].func) == cudaSuccess && b <= fa.maxThreadsPerBlock) {
      it->second = -it->second;
      *vi_out = vi;
      *block_out = b;
      return HISQ_OK;
    }
    cudaGetLastError();
    ctx->tune.erase(it);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HISQ_CUDA(cudaStreamIsCapturing(ctx->stream, &cap));
  if (!ctx->autotune || cap != cudaStreamCaptureStatusNone) {
    cudaFuncAttributes fa;
    HISQ_CUDA(cudaFuncGetAttributes(&fa, v[0].func));
    const int b = fa.maxThreadsPerBlock >= 256 ? 256 : 128;
    *vi_out = 0;
    *block_out = b;
    if (cap == cudaStreamCaptureStatusNone) ctx->tune[key] = b;
    return HISQ_OK;
  }
  // powers of two and the sizes between them: on small lattices a block size that spreads the
  // blocks evenly over the SMs matters
  static const int cands[] = {64, 96, 128, 160, 192, 224, 256, 384, 512};
  cudaEvent_t e0, e1;
  HISQ_CUDA(cudaEventCreate(&e0));
  HISQ_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_v = 0, best_b = 128;
  for (int i = 0; i < nv; ++i) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, v[i].func) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    for (int b : cands) {
      if (b > fa.maxThreadsPerBlock) continue;
      cudaError_t err = v[i].run(b);  // warm-up
      if (err != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < 3; ++r) v[i].run(b);
      note_launch(ctx, 4);
      cudaEventRecord(e1, ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_v = i;
        best_b = b;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HISQ_CUDA(cudaGetLastError());
  ctx->tune[key] = best_v * 10000 + best_b;
  *vi_out = best_v;
  *block_out = best_b;
  return HISQ_OK;
}

template <typename Run>
int tuned_block(hisq_ctx* ctx, const char* key, const void* func, Run run, int* block_out) {
  TuneVariant v{func, run};
  int vi = 0;
  return tuned_variant(ctx, key, &v, 1, &vi, block_out);
}

}  // namespace hisq
