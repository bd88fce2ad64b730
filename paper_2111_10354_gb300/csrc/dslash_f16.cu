// Dslash instantiations with FP16 links: FP16 spinors (storage-only 16-bit path) or FP32
// spinors (the mixed-precision CG's inner operator). FP32 arithmetic.
#include "dslash_launch.cuh"

namespace hisq {
int dslash_launch_f16(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_F16) return dslash_launch_t<__half, __half>(ctx, c);
  if (sp == HISQ_F32) return dslash_launch_t<__half, float>(ctx, c);
  return set_error(HISQ_EINVAL, "FP16 links pair with FP16 or FP32 spinors");
}
}  // namespace hisq
