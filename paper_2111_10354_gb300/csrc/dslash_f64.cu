// Dslash instantiations with FP64 links (FP64 spinors, FP64 arithmetic).
#include "dslash_launch.cuh"

namespace hisq {
int dslash_launch_f64(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_F64) return dslash_launch_t<double, double>(ctx, c);
  return set_error(HISQ_EINVAL, "FP64 links pair with FP64 spinors only");
}
}  // namespace hisq
