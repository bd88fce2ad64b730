// Interleaved multi-RHS Dslash instantiations with FP32 links (FP32 vectors, FP32 arithmetic).
#include "dslash_mrhs_launch.cuh"

namespace hisq {
int mrhs_launch_f32(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_F32) return mrhs_launch_t<float, float>(ctx, c);
  return set_error(HISQ_EINVAL, "FP32 links pair with FP32 vectors only");
}
}  // namespace hisq
