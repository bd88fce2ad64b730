// Host-side launcher of the Dslash kernel for one (link, spinor) precision pair: splits
// nrhs into groups that share each link read and picks the launch form and block size
// with the autotuner.
#pragma once
#include <string>

#include "dslash_impl.cuh"
#include "tune.h"

namespace hisq {

// Tile height (z-planes) of the tiled site walk for a launch reading nvec vectors of vbytes per site: the
// largest divisor of Lz whose seven-slice window of input vectors (the +-3 t-hops) stays within 24 MB, the
// part of L2 the gathers can count on while the links stream through. Where the natural order already
// fits, the largest proper divisor (the walk is then a form for the tuner to reject, and for the tests).
inline int walk_zb_for(const hisq_ctx* ctx, int nvec, size_t vbytes) {
  const Geom& g = ctx->g;
  const double plane_bytes = (double)g.half_x * g.L[1] * nvec * vbytes;
  const double budget = 24.0 * (1 << 20);
  int cap = (int)(budget / (7.0 * plane_bytes));
  if (cap >= g.L[2]) cap = g.L[2] / 2;
  int zb = 1;
  for (int d = 1; d <= cap && d <= g.L[2]; ++d)
    if (g.L[2] % d == 0) zb = d;
  return zb;
}

// The tiled walk's parameters in the kernel arguments (reciprocals for the kernel's two divisions).
inline void set_walk(const hisq_ctx* ctx, DslashKArgs& a, int zb) {
  a.walk_zb = zb;
  a.walk_chunk = zb * ctx->g.half_x * ctx->g.L[1];
  a.walk_m_chunk = ~0ull / (unsigned long long)a.walk_chunk + 1;
  a.walk_m_lt = ~0ull / (unsigned long long)ctx->g.L[3] + 1;
}

// One launch form: NR vectors per thread, TS threads per site (NR * TS vectors per launch); WALK: the
// output sites in the tiled walk (walk_zb_for) instead of cb order.
template <typename LR, typename SR, int NR, int EPI, bool COMP, int TS, bool WALK = false, bool PF = false>
static TuneVariant dslash_variant(hisq_ctx* ctx, const DslashKArgs& a) {
  // the launcher captures two pointers only, so std::function keeps it without a heap allocation
  return TuneVariant{(const void*)dslash_kernel<LR, SR, NR, EPI, COMP, TS, PF>, [ctx, &a](int block) -> cudaError_t {
                       int grid = (int)(((size_t)ctx->g.half * TS + block - 1) / block);
                       // Plain launches in cb order: a grid of two resident waves with a grid-stride loop.
                       // The tiled walk's plain launches take one site per thread: blocks are dispatched in
                       // index order, so the sites in flight slide through the walk instead of each
                       // resident wave of a grid-stride loop sweeping the whole lattice in turn (144^3x36:
                       // DRAM traffic 1.13x -> 1.02x of the algorithmic bytes). Reducing launches: one wave
                       // of the blocks that are resident together keeps the partials, and the finishing
                       // block's sum over them, short (a grid of one site per thread made the per-vector
                       // sums of the 8-vector form the launch's tail).
                       int cap = WALK ? grid : max_grid_blocks(ctx, block);
                       if (EPI == EPI_AXPY && a.partials) {
                         int per_sm = 0;
                         cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &per_sm, dslash_kernel<LR, SR, NR, EPI, COMP, TS, PF>, block, 0);
                         cap = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
                       }
                       if (grid > cap) grid = cap;
                       DslashKArgs b = a;
                       if (WALK) set_walk(ctx, b, walk_zb_for(ctx, NR * TS, 6 * sizeof(SR)));
                       return launch_dependent(ctx, dslash_kernel<LR, SR, NR, EPI, COMP, TS, PF>, grid, block, b);
                     }};
}

template <int N>
static int launch_tuned(hisq_ctx* ctx, const char* key, const TuneVariant (&v)[N]) {
  int vi = 0, block = 0;
  int rc = tuned_variant(ctx, key, v, N, &vi, &block);
  if (rc != HISQ_OK) return rc;
  HISQ_CUDA(v[vi].run(block));
  note_launch(ctx);
  return HISQ_OK;
}

// A group of nr vectors shares each link read. The launch forms differ in how the group is spread
// over threads (vectors per thread x threads per site); the tuner times each and keeps the fastest.
template <typename LR, typename SR, int EPI, bool COMP>
static int launch_nr(hisq_ctx* ctx, const DslashKArgs& a, int nr) {
  char key[64];
  snprintf(key, sizeof key, "dslash/l%d/s%d/nr%d/e%d/c%d", Real<LR>::prec, Real<SR>::prec, nr, EPI, (int)COMP);
  switch (nr) {
    case 1: {
      const TuneVariant v[] = {dslash_variant<LR, SR, 1, EPI, COMP, 1>(ctx, a),
                               dslash_variant<LR, SR, 1, EPI, COMP, 1, true>(ctx, a)};
      return launch_tuned(ctx, key, v);
    }
    case 2: {
      const TuneVariant v[] = {dslash_variant<LR, SR, 2, EPI, COMP, 1>(ctx, a),
                               dslash_variant<LR, SR, 1, EPI, COMP, 2>(ctx, a)};
      return launch_tuned(ctx, key, v);
    }
    case 4: {
      const TuneVariant v[] = {dslash_variant<LR, SR, 4, EPI, COMP, 1>(ctx, a),
                               dslash_variant<LR, SR, 2, EPI, COMP, 2>(ctx, a),
                               dslash_variant<LR, SR, 1, EPI, COMP, 4>(ctx, a)};
      return launch_tuned(ctx, key, v);
    }
    case 8:
      if constexpr (sizeof(LR) < 8) {
        const TuneVariant v[] = {dslash_variant<LR, SR, 8, EPI, COMP, 1>(ctx, a),
                                 dslash_variant<LR, SR, 4, EPI, COMP, 2>(ctx, a),
                                 dslash_variant<LR, SR, 2, EPI, COMP, 4>(ctx, a),
                                 dslash_variant<LR, SR, 8, EPI, COMP, 1, true>(ctx, a),
                                 dslash_variant<LR, SR, 4, EPI, COMP, 2, true>(ctx, a),
                                 dslash_variant<LR, SR, 2, EPI, COMP, 4, true>(ctx, a),
                                 dslash_variant<LR, SR, 8, EPI, COMP, 1, false, true>(ctx, a),
                                 dslash_variant<LR, SR, 8, EPI, COMP, 1, true, true>(ctx, a)};
        return launch_tuned(ctx, key, v);
      }
      break;
  }
  return set_error(HISQ_EINVAL, "unsupported rhs group %d", nr);
}

// Largest rhs group per launch (register budget): FP64 4, others 8 -- a group of 16 needs more
// than the 255 registers a thread can hold and spills (measured 5x slower than two groups of 8).
template <typename LR>
static int max_group() {
  return sizeof(LR) == 8 ? 4 : 8;
}

template <typename LR, typename SR>
int dslash_launch_t(hisq_ctx* ctx, const DslashCall& c) {
  const size_t site_bytes = 6 * sizeof(SR);
  const int gmax = max_group<LR>();
  int r0 = 0;
  while (r0 < c.nrhs) {
    const int left = c.nrhs - r0;
    int nr = 1;
    while (nr * 2 <= left && nr * 2 <= gmax) nr *= 2;
    DslashKArgs a;
    a.g = ctx->g;
    a.links = ctx->links[Real<LR>::prec];
    a.blk_bytes = link_block_bytes(Real<LR>::prec, ctx->g.half);
    a.out_parity = c.out_parity;
    a.out = (char*)c.out + (size_t)r0 * c.rhs_stride * site_bytes;
    a.in = (const char*)c.in + (size_t)r0 * c.rhs_stride * site_bytes;
    a.rhs_stride = c.rhs_stride;
    a.y = c.y ? (const char*)c.y + (size_t)r0 * c.rhs_stride * site_bytes : nullptr;
    for (int r = 0; r < 16; ++r) a.a[r] = (c.a_rhs && r0 + r < c.nrhs) ? c.a_rhs[r0 + r] : c.a;
    a.partials = c.partials ? c.partials + (size_t)r0 * partial_stride(ctx) : nullptr;
    a.dot_out = c.dot_out ? c.dot_out + r0 : nullptr;
    a.counter = c.counter;
    a.skip = c.skip;
    // compressed long links (two rows, third reconstructed) whenever the context keeps them
    const bool comp = sizeof(LR) < 8 && ctx->naik != 0.0 && ctx->long12[Real<LR>::prec] != nullptr;
    a.long12 = comp ? ctx->long12[Real<LR>::prec] : nullptr;
    a.blk12 = long12_block_bytes(Real<LR>::prec, ctx->g.half);
    a.inv_naik = comp ? (float)(1.0 / ctx->naik) : 0.f;
    a.flags = ctx->load_flags;
    int rc;
    if constexpr (sizeof(LR) < 8) {
      if (comp)
        rc = c.epi == EPI_PLAIN ? launch_nr<LR, SR, EPI_PLAIN, true>(ctx, a, nr)
                                : launch_nr<LR, SR, EPI_AXPY, true>(ctx, a, nr);
      else
        rc = c.epi == EPI_PLAIN ? launch_nr<LR, SR, EPI_PLAIN, false>(ctx, a, nr)
                                : launch_nr<LR, SR, EPI_AXPY, false>(ctx, a, nr);
    } else {
      rc = c.epi == EPI_PLAIN ? launch_nr<LR, SR, EPI_PLAIN, false>(ctx, a, nr)
                              : launch_nr<LR, SR, EPI_AXPY, false>(ctx, a, nr);
    }
    if (rc != HISQ_OK) return rc;
    r0 += nr;
  }
  return HISQ_OK;
}

}  // namespace hisq
