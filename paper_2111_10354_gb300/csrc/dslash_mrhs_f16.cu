// Interleaved multi-RHS Dslash instantiations with FP16 links: FP16 vectors (16-bit storage) or FP32
// vectors (the mixed-precision CG's inner operator). FP32 arithmetic.
#include "dslash_mrhs_launch.cuh"

namespace hisq {
int mrhs_launch_f16(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_F16) return mrhs_launch_t<__half, __half>(ctx, c);
  if (sp == HISQ_F32) return mrhs_launch_t<__half, float>(ctx, c);
  return set_error(HISQ_EINVAL, "FP16 links pair with FP16 or FP32 vectors");
}
}  // namespace hisq
