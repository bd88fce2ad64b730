// Dslash instantiations with double-float links: FP64 vectors at the boundary, converted to
// double-float as they are read, double-float arithmetic, FP64 output.
#include "dslash_launch.cuh"

namespace hisq {
int dslash_launch_df64(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_F64 || sp == HISQ_DF64) return dslash_launch_t<df64, double>(ctx, c);
  return set_error(HISQ_EINVAL, "double-float links pair with FP64 vectors only");
}
}  // namespace hisq
