// HISQ even/odd Dslash kernel (the stencil that dominates the time of the CG, Sec. 3): for each
// output site x of one parity,
//   out(x) = sum_mu [ F_mu(x) in(x+mu) - F_mu(x-mu)^dag in(x-mu)
//                   + L_mu(x) in(x+3mu) - L_mu(x-3mu)^dag in(x-3mu) ]
// with staggered phases and the antiperiodic-t sign already folded into F and L.
//
// Design: one thread (or TS threads) per output site (grid-stride), NR right-hand sides per
// thread so every link is read from HBM once per launch however many vectors it is applied to
// (the multi-RHS form, Sec. 3). Links stream through 16-byte no-L1-allocate loads from
// their chunk planes; neighbour vectors go through L1/L2, where the 16-fold reuse of
// each input site is served. Accumulation is FP64 for FP64 storage and FP32 otherwise.
#pragma once
#include <type_traits>

#include "internal.cuh"
#include "pdl.cuh"
#include "reduce_warp.cuh"

namespace hisq {

template <typename T>
__device__ __forceinline__ void cmac_conj_sub(cplx<T>& acc, const cplx<T>& a, const cplx<T>& b) {
  // acc -= conj(a) * b
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

// acc -= conj(a) * b in double-float on lane pairs: (re, im) += (-a.re, -a.re) (b.re, b.im)
// + (-a.im, a.im) (b.im, b.re).
__device__ __forceinline__ void cmac_conj_sub(cplx<df64>& acc, const cplx<df64>& a, const cplx<df64>& b) {
  df64x2 c{make_float2(acc.re.hi, acc.im.hi), make_float2(acc.re.lo, acc.im.lo)};
  c = df2_fma({make_float2(-a.re.hi, -a.re.hi), make_float2(-a.re.lo, -a.re.lo)},
              {make_float2(b.re.hi, b.im.hi), make_float2(b.re.lo, b.im.lo)}, c);
  c = df2_fma({make_float2(-a.im.hi, a.im.hi), make_float2(-a.im.lo, a.im.lo)},
              {make_float2(b.im.hi, b.re.hi), make_float2(b.im.lo, b.re.lo)}, c);
  acc.re = df64(c.hi.x, c.lo.x);
  acc.im = df64(c.hi.y, c.lo.y);
}

struct DslashKArgs {
  Geom g;
  const char* links;  // resident link storage of the link precision (16 blocks)
  size_t blk_bytes;   // bytes of one link block
  int out_parity;
  void* out;
  const void* in;
  size_t rhs_stride;  // sites between consecutive rhs vectors
  const void* y;      // EPI_AXPY
  double a[16];       // per-rhs diagonal coefficient 4m^2 + sigma_r
  double* partials;   // [NR][gridDim.x]
  double* dot_out;    // [NR]
  unsigned* counter;
  const int* skip;    // when non-null and set: a finished solver cycle, do nothing
  const char* long12;  // compressed long links (COMP variants)
  size_t blk12;
  float inv_naik;
  unsigned flags;      // load flags: phases / antiperiodic t (fold signs of compressed links)
  int walk_zb = 0;     // > 0: output sites walked in tiles of walk_zb z-planes (see walk_cb)
  int walk_chunk = 0;  // walk_zb * Lx Ly / 2: cb numbers per (tile, t) chunk
  unsigned long long walk_m_chunk = 0, walk_m_lt = 0;  // 2^64 / walk_chunk and 2^64 / Lt, rounded up
};

// Output site of walk position w when the sites are walked in tiles of zb z-planes: tile by tile, and in
// a tile t-slice by t-slice, each (tile, t) chunk being zb * Lx Ly / 2 consecutive cb numbers. In the
// natural order the +-1 and +-3 t-neighbours of the sites in flight span seven whole t-slices of the
// input vectors, which exceeds L2 on large lattices (144^3x36 FP32: 250 MB); in the tiled walk they span
// seven slices of one tile. The neighbours across a tile's z faces are the ones read again. The two
// divisions are multiplications by rounded-up reciprocals (exact for w < 2^30 and divisors < 2^34).
__device__ __forceinline__ int walk_cb(const Geom& g, const DslashKArgs& k, int w) {
  const int q = (int)__umul64hi((unsigned long long)w, k.walk_m_chunk);  // (tile, t) chunk
  const int o = w - q * k.walk_chunk;
  const int tile = (int)__umul64hi((unsigned long long)q, k.walk_m_lt);
  const int t = q - tile * g.L[3];
  return (tile * k.walk_zb + g.L[2] * t) * (g.half_x * g.L[1]) + o;
}

// What the compressed-long-link path needs at one site.
struct Comp12 {
  const char* long12;
  size_t blk12;
  float inv_naik;
  unsigned flags;
};

// Requests for data a later hop reads: the vectors into L1, the (streamed, evict-first) link into L2.
// Hints only: nothing waits on them and no register receives data.
__device__ __forceinline__ void prefetch_l1(const void* a) { asm volatile("prefetch.global.L1 [%0];" ::"l"(a)); }
__device__ __forceinline__ void prefetch_l2(const void* a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); }
// The link of site cb in block blk, plane by plane as LinkIO reads it (FP32: 4 x 16 B + 8 B; 16-bit:
// 2 x 16 B + 4 B); the 8-vector forms that prefetch exist for these precisions only.
template <typename LR>
__device__ __forceinline__ void prefetch_link(const char* blk, int half, int cb) {
  if constexpr (std::is_same<LR, float>::value) {
#pragma unroll
    for (int j = 0; j < 4; ++j) prefetch_l2(blk + ((size_t)j * half + cb) * 16);
    prefetch_l2(blk + (size_t)64 * half + (size_t)cb * 8);
  } else if constexpr (sizeof(LR) == 2) {
#pragma unroll
    for (int j = 0; j < 2; ++j) prefetch_l2(blk + ((size_t)j * half + cb) * 16);
    prefetch_l2(blk + (size_t)32 * half + (size_t)cb * 4);
  }
}

// The 16 hopping terms at output site cb (parity p) for NR vectors: acc[r][i] = (D in_r)(x)_i.
// links: the 16 blocks of one lattice in the link precision; in: NR vectors rhs_stride sites apart.
// pf (8-vector forms): while a hop computes, the next hop's NR vectors are requested into L1 and its
// link into L2, so the next hop's loads do not wait on DRAM (16 warps per SM at 128 registers leave
// little else to cover that latency).
template <typename LR, typename SR, int NR, bool COMP = false>
__device__ __forceinline__ void dslash_site(const Geom& g, const char* links, size_t blk_bytes, int p, int cb,
                                            const void* in, size_t rhs_stride,
                                            cplx<typename Real<LR>::acc> (&acc)[NR][3], const Comp12& cz = Comp12{},
                                            bool pf = false) {
  using A = typename Real<LR>::acc;
  using SA = typename Real<SR>::acc;
  const char* fwd = links + (size_t)(p * 8) * blk_bytes;        // blocks of parity p
  const char* bwd = links + (size_t)((1 - p) * 8) * blk_bytes;  // blocks of parity 1-p
  int c[4];
  site_coords(g, p, cb, c);
  const int idx = lex_index(g, c);
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[r][i] = {A(0), A(0)};

  // groups of 8 vectors keep the direction loop rolled: the fully unrolled body (16 hops x 8 vectors)
  // outgrows the instruction cache and the warps stall on instruction fetch (48^3x12 FP32: 260 -> 245 us;
  // FP16: 204 -> 183 us); at 4 vectors the unrolled body is faster (156 vs 171 us)
  // double-float keeps it rolled as well (its hoisted link loads otherwise exceed the register budget)
  constexpr int MU_UNROLL = (NR >= 8 || std::is_same<LR, df64>::value) ? 1 : 4;
#pragma unroll MU_UNROLL
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int kind = 0; kind < 2; ++kind) {
      const int hop = kind == 0 ? 1 : 3;
      const char* blk_f = fwd + (size_t)(kind * 4 + mu) * blk_bytes;
      const char* blk_b = bwd + (size_t)(kind * 4 + mu) * blk_bytes;
      // forward hop: + W_mu(x) in(x + hop mu)
      {
        const int nb = neighbour_cb(g, c, idx, mu, +hop);
        if constexpr (NR >= 8 && sizeof(LR) < 8) {
          if (pf) {  // the backward hop of this (mu, kind)
            constexpr size_t VB = 6 * sizeof(SR);  // bytes of one vector at one site
            const int nbb = neighbour_cb(g, c, idx, mu, -hop);
#pragma unroll
            for (int r = 0; r < NR; ++r) prefetch_l1((const char*)in + ((size_t)r * rhs_stride + nbb) * VB);
            if (!(COMP && kind == 1)) prefetch_link<LR>(blk_b, g.half, nbb);
          }
        }
        cplx<A> U[9];
        if constexpr (COMP && sizeof(LR) < 8) {
          if (kind == 1) {
            Link12IO<LR>::load(cz.long12 + (size_t)(p * 4 + mu) * cz.blk12, g.half, cb, U);
            const int sg = folded_long_sign(g, cz.flags, mu, c[0], c[1], c[2], c[3]);
            reconstruct_row2(U, A(sg) * A(cz.inv_naik));
          } else {
            LinkIO<LR>::load(blk_f, g.half, cb, U);
          }
        } else {
          LinkIO<LR>::load(blk_f, g.half, cb, U);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          cplx<SA> vs[3];
          VecIO<SR>::load(in, (size_t)r * rhs_stride + nb, vs);
          cplx<A> v[3] = {{A(vs[0].re), A(vs[0].im)}, {A(vs[1].re), A(vs[1].im)}, {A(vs[2].re), A(vs[2].im)}};
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) cmac(acc[r][i], U[3 * i + j], v[j]);
        }
      }
      // backward hop: - W_mu(x - hop mu)^dag in(x - hop mu)
      {
        const int nb = neighbour_cb(g, c, idx, mu, -hop);
        if constexpr (NR >= 8 && sizeof(LR) < 8) {
          if (pf && (kind == 0 || mu < 3)) {  // the forward hop of the next (mu, kind)
            constexpr size_t VB = 6 * sizeof(SR);
            const int kn = kind ^ 1, mn = kind == 0 ? mu : mu + 1;
            const int nbn = neighbour_cb(g, c, idx, mn, kn == 0 ? 1 : 3);
#pragma unroll
            for (int r = 0; r < NR; ++r) prefetch_l1((const char*)in + ((size_t)r * rhs_stride + nbn) * VB);
            if (!(COMP && kn == 1)) prefetch_link<LR>(fwd + (size_t)(kn * 4 + mn) * blk_bytes, g.half, cb);
          }
        }
        cplx<A> U[9];
        if constexpr (COMP && sizeof(LR) < 8) {
          if (kind == 1) {
            Link12IO<LR>::load(cz.long12 + (size_t)((1 - p) * 4 + mu) * cz.blk12, g.half, nb, U);
            // the link sits at y = x - 3mu: only its t coordinate can change the fold sign
            const int yt = mu == 3 ? (c[3] >= 3 ? c[3] - 3 : c[3] - 3 + g.L[3]) : c[3];
            const int sg = folded_long_sign(g, cz.flags, mu, c[0], c[1], c[2], yt);
            reconstruct_row2(U, A(sg) * A(cz.inv_naik));
          } else {
            LinkIO<LR>::load(blk_b, g.half, nb, U);
          }
        } else {
          LinkIO<LR>::load(blk_b, g.half, nb, U);
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          cplx<SA> vs[3];
          VecIO<SR>::load(in, (size_t)r * rhs_stride + nb, vs);
          cplx<A> v[3] = {{A(vs[0].re), A(vs[0].im)}, {A(vs[1].re), A(vs[1].im)}, {A(vs[2].re), A(vs[2].im)}};
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) cmac_conj_sub(acc[r][i], U[3 * j + i], v[j]);
        }
      }
    }
  }
}

// Register budget: the single-vector FP32/16-bit kernels are held to 64 registers (4 blocks of 256
// per SM): the fused epilogue otherwise grows to ~100 registers and halves the resident warps,
// which for this memory-bound stencil halves the bandwidth. FP64 keeps its registers (it is
// bound by GB300's FP64 pipe, and a 64-register cap spills).
template <typename LR, int NR>
struct DslashBounds {
  static constexpr int threads = NR == 1 ? (sizeof(LR) < 8 ? 256 : 512) : (NR == 2 ? 512 : (NR == 4 ? 256 : 128));
  // FP32/16-bit: 64 registers for one vector, 128 for groups of 4 and 8 (enough warps in flight)
  static constexpr int min_blocks = sizeof(LR) == 8 ? 1 : (NR == 1 ? 4 : (NR == 2 ? 1 : (NR == 4 ? 2 : (NR == 8 ? 4 : 1))));
};
// Double-float: 128 registers for one vector (a double-float link is 36 registers), all 255 for
// groups, where fewer spill.
template <int NR>
struct DslashBounds<df64, NR> {
  static constexpr int threads = NR == 1 ? 256 : 128;
  static constexpr int min_blocks = NR == 1 ? 2 : 1;
};

// TS threads share one output site, each applying its links to NR of the site's NR*TS vectors
// (thread sub = threadIdx.x % TS takes vectors sub*NR .. sub*NR+NR-1). The TS lanes of a site sit in
// one warp and load the same link words in the same instruction, so a link still leaves HBM once
// per launch, while each thread holds fewer accumulators (more warps in flight per SM).
// PF: the 8-vector forms that prefetch each next hop (a template parameter, so the other forms carry
// none of its code or registers).
template <typename LR, typename SR, int NR, int EPI, bool COMP = false, int TS = 1, bool PF = false>
__global__ void __launch_bounds__(DslashBounds<LR, NR>::threads, DslashBounds<LR, NR>::min_blocks)
    dslash_kernel(const DslashKArgs k) {
  using A = typename Real<LR>::acc;  // accumulation type follows the link precision
  using SA = typename Real<SR>::acc;
  static_assert(TS == 1 || TS == 2 || TS == 4, "threads per site");
  griddep_wait();  // a programmatic dependent launch (pdl.cuh): nothing is touched before this
  griddep_launch_dependents();
  if (k.skip && *k.skip) return;  // uniform over the grid
  const Geom& g = k.g;
  const int p = k.out_parity;
  double dot[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) dot[r] = 0.0;
  const int sub = TS == 1 ? 0 : (int)(threadIdx.x % TS);  // blockDim.x is a multiple of TS
  const int rbase = sub * NR;
  const size_t vbytes = (size_t)rbase * k.rhs_stride * 6 * sizeof(SR);
  const void* in = (const char*)k.in + vbytes;
  void* out = (char*)k.out + vbytes;
  const void* y = k.y ? (const void*)((const char*)k.y + vbytes) : nullptr;

  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) / TS; w < g.half; w += gridDim.x * blockDim.x / TS) {
    const int cb = k.walk_zb ? walk_cb(g, k, w) : w;
    cplx<A> acc[NR][3];
    dslash_site<LR, SR, NR, COMP>(g, k.links, k.blk_bytes, p, cb, in, k.rhs_stride, acc,
                                  Comp12{k.long12, k.blk12, k.inv_naik, k.flags}, PF);

#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const size_t site = (size_t)r * k.rhs_stride + cb;
      cplx<SA> o[3];
      if (EPI == EPI_PLAIN) {
#pragma unroll
        for (int i = 0; i < 3; ++i) o[i] = {SA(acc[r][i].re), SA(acc[r][i].im)};
      } else {
        // the axpy in the accumulation type (FP64 for double-float: one FMA per entry)
        using EA = typename std::conditional<std::is_same<A, df64>::value, double, A>::type;
        cplx<SA> yv[3];
        VecIO<SR>::load(y, site, yv);
        const EA a = EA(k.a[rbase + r]);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          o[i].re = SA(fma(a, EA(yv[i].re), -EA(acc[r][i].re)));
          o[i].im = SA(fma(a, EA(yv[i].im), -EA(acc[r][i].im)));
        }
        if (k.partials) {
          // the site's term in the arithmetic precision, summed over sites in FP64 (GB300's
          // FP64 pipe is ~2 ops/clk/SM: one conversion and one add per site, not twelve)
          SA t = SA(0);
#pragma unroll
          for (int i = 0; i < 3; ++i) t += yv[i].re * o[i].re + yv[i].im * o[i].im;
          dot[r] += (double)t;
        }
      }
      VecIO<SR>::store(out, site, o);
    }
  }

  if (EPI == EPI_AXPY) {
    if (k.partials == nullptr) return;  // uniform over the grid
    __shared__ double red[32];
#pragma unroll
    for (int R = 0; R < NR * TS; ++R) {
      double s = block_sum_dyn(sub == R / NR ? dot[R % NR] : 0.0, red);
      if (threadIdx.x == 0) k.partials[(size_t)R * gridDim.x + blockIdx.x] = s;
    }
    if (last_block_done(k.counter)) {
      if constexpr (NR * TS == 1) {
        double s = sum_partials_dyn(k.partials, gridDim.x, red);
        if (threadIdx.x == 0) k.dot_out[0] = s;
      } else {
        // several vectors: one warp per vector sums its partials, the vectors' sums in parallel
        const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int R = threadIdx.x >> 5; R < NR * TS; R += nw) {
          const double s = warp_sum_partials(k.partials + (size_t)R * gridDim.x, gridDim.x);
          if (lane == 0) k.dot_out[R] = s;
        }
      }
    }
  }
}

}  // namespace hisq
