// Interleaved multi-RHS Dslash instantiations with FP64 links (FP64 arithmetic) and with double-float
// links (FP64 vectors converted to double-float as they are read, double-float arithmetic).
#include "dslash_mrhs_launch.cuh"

namespace hisq {
int mrhs_launch_f64(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_F64) return mrhs_launch_t<double, double>(ctx, c);
  return set_error(HISQ_EINVAL, "FP64 links pair with FP64 vectors only");
}
int mrhs_launch_df64(hisq_ctx* ctx, int sp, const DslashCall& c) {
  if (sp == HISQ_F64 || sp == HISQ_DF64) return mrhs_launch_t<df64, double>(ctx, c);
  return set_error(HISQ_EINVAL, "double-float links pair with FP64 vectors only");
}
}  // namespace hisq
