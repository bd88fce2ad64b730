// Host-side launcher of the interleaved multi-RHS Dslash for one (link, spinor) precision pair:
// one launch covers all N vectors; the autotuner picks the granules per thread and the block size.
#pragma once
#include <stdio.h>

#include "dslash_mrhs.cuh"
#include "tune.h"

namespace hisq {

inline int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// One launch form: NG granules per thread, ts = the next power of two of ceil(ngr / NG) threads per site.
template <int NG>
inline int mrhs_ts(int ngr) {
  return next_pow2((ngr + NG - 1) / NG);
}

template <typename LR, typename SR, int NG, int EPI, bool COMP>
static TuneVariant mrhs_variant(hisq_ctx* ctx, const MrhsArgs& a) {
  return TuneVariant{(const void*)dslash_mrhs_kernel<LR, SR, NG, EPI, COMP>, [ctx, &a](int block) -> cudaError_t {
                       MrhsArgs b = a;
                       b.ts = mrhs_ts<NG>(a.ngr);
                       if (block % b.ts) return cudaErrorInvalidConfiguration;
                       int grid = (int)(((size_t)ctx->g.half * b.ts + block - 1) / block);
                       int cap = max_grid_blocks(ctx, block);
                       if (EPI == EPI_AXPY && a.partials) {
                         // reducing launches: one wave of co-resident blocks keeps the partials short
                         int per_sm = 0;
                         cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &per_sm, dslash_mrhs_kernel<LR, SR, NG, EPI, COMP>, block, 0);
                         cap = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
                       }
                       if (grid > cap) grid = cap;
                       dslash_mrhs_kernel<LR, SR, NG, EPI, COMP><<<grid, block, 0, ctx->stream>>>(b);
                       return cudaGetLastError();
                     }};
}

// The launch forms for ngr granules per site: NG granules per thread with at most 32 threads per site
// (a site's threads stay in one warp), and no form whose threads would mostly idle (NG > ngr).
template <typename LR, typename SR, int EPI, bool COMP>
static int mrhs_launch_forms(hisq_ctx* ctx, const MrhsArgs& a, const char* key) {
  const int ngr = a.ngr;
  TuneVariant v[3];
  int nv = 0;
  if (mrhs_ts<1>(ngr) <= 32) v[nv++] = mrhs_variant<LR, SR, 1, EPI, COMP>(ctx, a);
  if (ngr >= 2 && mrhs_ts<2>(ngr) <= 32) v[nv++] = mrhs_variant<LR, SR, 2, EPI, COMP>(ctx, a);
  // four granules per thread only where they are four FP32 granules (8 vectors): 16 vectors of 16-bit
  // storage spill
  if constexpr (std::is_same<SR, float>::value) {
    if (ngr >= 4) v[nv++] = mrhs_variant<LR, SR, 4, EPI, COMP>(ctx, a);
  }
  if (nv == 0) return set_error(HISQ_EINVAL, "no launch form for %d granules per site", ngr);
  int vi = 0, block = 0;
  int rc = tuned_variant(ctx, key, v, nv, &vi, &block);
  if (rc != HISQ_OK) return rc;
  HISQ_CUDA(v[vi].run(block));
  note_launch(ctx);
  return HISQ_OK;
}

// D on the interleaved layout: c.nrhs vectors per site ([cb][color][rhs]), all in one launch.
template <typename LR, typename SR>
int mrhs_launch_t(hisq_ctx* ctx, const DslashCall& c) {
  constexpr int G = GranIO<SR>::G;
  if (c.nrhs < 1 || c.nrhs > MRHS_MAX || c.nrhs % G)
    return set_error(HISQ_EINVAL, "interleaved layout: %d vectors per site is not a multiple of %d in [1, %d]", c.nrhs,
                     G, MRHS_MAX);
  MrhsArgs a;
  a.g = ctx->g;
  a.links = ctx->links[Real<LR>::prec];
  a.blk_bytes = link_block_bytes(Real<LR>::prec, ctx->g.half);
  a.out_parity = c.out_parity;
  a.out = c.out;
  a.in = c.in;
  a.ngr = c.nrhs / G;
  a.ts = 1;
  a.y = c.y;
  for (int r = 0; r < MRHS_MAX; ++r) a.a[r] = (c.a_rhs && r < c.nrhs) ? c.a_rhs[r] : c.a;
  a.partials = c.partials;
  a.dot_out = c.dot_out;
  a.counter = c.counter;
  a.skip = c.skip;
  const bool comp = sizeof(LR) < 8 && ctx->naik != 0.0 && ctx->long12[Real<LR>::prec] != nullptr;
  a.long12 = comp ? ctx->long12[Real<LR>::prec] : nullptr;
  a.blk12 = long12_block_bytes(Real<LR>::prec, ctx->g.half);
  a.inv_naik = comp ? (float)(1.0 / ctx->naik) : 0.f;
  a.flags = ctx->load_flags;
  char key[64];
  snprintf(key, sizeof key, "mrhs/l%d/s%d/n%d/e%d/c%d", Real<LR>::prec, Real<SR>::prec, c.nrhs, c.epi, (int)comp);
  if constexpr (sizeof(LR) < 8) {
    if (comp)
      return c.epi == EPI_PLAIN ? mrhs_launch_forms<LR, SR, EPI_PLAIN, true>(ctx, a, key)
                                : mrhs_launch_forms<LR, SR, EPI_AXPY, true>(ctx, a, key);
  }
  return c.epi == EPI_PLAIN ? mrhs_launch_forms<LR, SR, EPI_PLAIN, false>(ctx, a, key)
                            : mrhs_launch_forms<LR, SR, EPI_AXPY, false>(ctx, a, key);
}

}  // namespace hisq
