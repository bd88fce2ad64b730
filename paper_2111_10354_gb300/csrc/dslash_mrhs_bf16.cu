// Interleaved multi-RHS Dslash instantiations with BF16 links: BF16 vectors (16-bit storage) or FP32
// vectors (the mixed-precision CG's inner operator). FP32 arithmetic.
#include "dslash_mrhs_launch.cuh"

namespace hisq {
int mrhs_launch_bf16(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_BF16) return mrhs_launch_t<__nv_bfloat16, __nv_bfloat16>(ctx, c);
  if (sp == HISQ_F32) return mrhs_launch_t<__nv_bfloat16, float>(ctx, c);
  return set_error(HISQ_EINVAL, "BF16 links pair with BF16 or FP32 vectors");
}
}  // namespace hisq
