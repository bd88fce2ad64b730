// CG on A = 4 m^2 - D_eo D_oe (Sec. 2 module list: CG with multi-RHS and mixed-precision
// variants; Sec. 3: the CG that takes about 60% of HISQ RHMC time).
//
// One iteration, for every rhs r at once:
//   t     = D_oe p                                   (Dslash, odd output)
//   Ap    = 4m^2 p - D_eo t,  pAp = Re<p, Ap>         (Dslash with fused axpy + FP64 dot)
//   alpha = rr / pAp;  x += alpha*scale*p;  r -= alpha*Ap;  rr' = |r|^2  \  one cooperative launch
//   beta  = rr' / rr;  p = r + beta*p;  rr = rr'; convergence flags     /   (k_cg_update)
// Plain FP64 CG keeps r, p, Ap in FP64 with FP64 links. Mixed precision keeps r, p, Ap in
// FP32 (or in the links' 16-bit format, on request) with links in the inner precision (FP32,
// FP16 or BF16 storage) and FP32 arithmetic; x, the reductions and the reliable update
// r = b - A x (FP64 links) stay FP64. Reliable
// update (a reading of the paper's "mixed precision" CG, which it names without detail):
// every reliable_period inner iterations, or as soon as the inner residual says the
// tolerance is met, recompute the true residual in FP64, rescale it to unit RMS entry,
// and restart the search direction from it (p = r). Keeping the old direction would pair
// alpha = |r_true|^2 / <p, A p> with a p built from the drifted iterated residual, which
// overshoots whenever the low-precision operator has let the two residuals part.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <cmath>
#include <type_traits>
#include <vector>

#include "solver_common.cuh"
#include "reduce_warp.cuh"
#include "trace.h"
#include "tune.h"

namespace hisq {

int dslash_launch(hisq_ctx* ctx, int lp, int sp, const DslashCall& c);
double dslash_bytes(const hisq_ctx* ctx, int lp, int sp, int nrhs);
bool is_device_ptr(const void* p);

// ------------------------------------------------------------------ kernels
// r = b - Ax (all FP64); rr_true = |r|^2; with init, bb = |b|^2.
__global__ void k_residual(const double2* __restrict__ b, size_t b_stride, const double2* __restrict__ Ax,
                           double2* __restrict__ r, size_t n /* complex entries per rhs */, SolverState* st,
                           double* partials, size_t pstride, unsigned* counter, int init) {
  const int rh = blockIdx.y;
  const size_t off = (size_t)rh * n;
  const double2* bq = b + (size_t)rh * b_stride;
  double v[2] = {0.0, 0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 bv = bq[i], av = Ax[off + i];
    double2 rv = make_double2(bv.x - av.x, bv.y - av.y);
    r[off + i] = rv;
    v[0] += rv.x * rv.x + rv.y * rv.y;
    v[1] += bv.x * bv.x + bv.y * bv.y;
  }
  double out[2][MAXR];
  if (grid_reduce<2>(v, partials, pstride, counter, out, st->nrhs) && threadIdx.x == 0) {
    for (int q = 0; q < st->nrhs; ++q) {
      st->rr_true[q] = out[0][q];
      if (init) st->bb[q] = out[1][q];
      if (!isfinite(out[0][q])) st->nonfinite = 1;
    }
  }
}

// |x_r|^2 per rhs into out[r] (detects a zero initial guess, whose residual is b itself).
__global__ void k_xnorm(const double2* __restrict__ x, size_t n, int nrhs, double* partials, size_t pstride,
                        unsigned* counter, double* out) {
  const int rh = blockIdx.y;
  const size_t off = (size_t)rh * n;
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 xv = x[off + i];
    v[0] += xv.x * xv.x + xv.y * xv.y;
  }
  double o[1][MAXR];
  if (grid_reduce<1>(v, partials, pstride, counter, o, nrhs) && threadIdx.x == 0)
    for (int q = 0; q < nrhs; ++q) out[q] = o[0][q];
}

// r = b (zero initial guess): rr_true = bb = |b|^2 without applying A.
__global__ void k_residual_zero(const double2* __restrict__ b, size_t b_stride, double2* __restrict__ r, size_t n,
                                SolverState* st, double* partials, size_t pstride, unsigned* counter) {
  const int rh = blockIdx.y;
  const size_t off = (size_t)rh * n;
  const double2* bq = b + (size_t)rh * b_stride;
  double v[1] = {0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 bv = bq[i];
    r[off + i] = bv;
    v[0] += bv.x * bv.x + bv.y * bv.y;
  }
  double o[1][MAXR];
  if (grid_reduce<1>(v, partials, pstride, counter, o, st->nrhs) && threadIdx.x == 0)
    for (int q = 0; q < st->nrhs; ++q) {
      st->rr_true[q] = o[0][q];
      st->bb[q] = o[0][q];
      if (!isfinite(o[0][q])) st->nonfinite = 1;
    }
}

// Bookkeeping of a reliable update (one thread): per-rhs verification, rescaling and the new cycle.
__device__ __forceinline__ void reliable_commit(SolverState* st, size_t n) {
  // the search direction restarts: the Lanczos relation of rhs 0's coefficients ends here
  if (st->lanczos && st->lanczos_n > 0 && st->lanczos_n < st->lanczos_cap && st->lanczos[st->lanczos_n - 1] != 0.0)
    st->lanczos[st->lanczos_n++] = 0.0;
  bool all = true;
  for (int q = 0; q < st->nrhs; ++q) {
    const bool c = st->rr_true[q] <= st->tol2[q];
    st->rhs_conv[q] = c;
    st->rhs_done[q] = c;
    const double s = sqrt(st->rr_true[q] / (double)n);
    if (!c && s > 0.0) {
      st->scale[q] = s;
      st->rr[q] = st->rr_true[q] / (s * s);
    }
    all = all && c;
  }
  st->done = all ? 1 : 0;
  st->cycle_iter = 0;
}

// Reliable update: for each rhs not yet verified, r_lo = r_hi / s (s = RMS entry of r_hi),
// p = r_lo (restart); rr = |r_hi|^2 / s^2. Verified rhs are frozen.
template <typename S>
__global__ void k_reliable(const double2* __restrict__ r_hi, S* __restrict__ r_lo, S* __restrict__ p, size_t n,
                           SolverState* st, int first, unsigned* counter) {
  const int rh = blockIdx.y;
  const size_t off = (size_t)rh * n;
  const bool conv = st->rr_true[rh] <= st->tol2[rh];
  const double s_new = sqrt(st->rr_true[rh] / (double)n);
  (void)first;
  if (!conv && s_new > 0.0) {
    const double inv = 1.0 / s_new;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      double2 rv = r_hi[off + i];
      const S re = S(rv.x * inv), im = S(rv.y * inv);
      r_lo[2 * (off + i)] = re;
      r_lo[2 * (off + i) + 1] = im;
      p[2 * (off + i)] = re;
      p[2 * (off + i) + 1] = im;
    }
  }
  if (last_block_done(counter) && threadIdx.x == 0) reliable_commit(st, n);
}


// Flat 16-byte access to vectors of complex entries for the BLAS kernels: the updates are
// entry-wise, so a thread takes Chunk<S>::K consecutive complex entries (one 16-byte load per
// vector; FP32 2, FP64 1) regardless of site boundaries. A rhs holds 3 * half complex
// entries, a multiple of 24, so chunks never straddle two rhs.
template <typename S>
struct Chunk;
template <>
struct Chunk<float> {
  static constexpr int K = 2;
  __device__ __forceinline__ static void load(const float* v, size_t c, cplx<float> o[2]) {
    const float4 w = reinterpret_cast<const float4*>(v)[c];
    o[0] = {w.x, w.y};
    o[1] = {w.z, w.w};
  }
  __device__ __forceinline__ static void store(float* v, size_t c, const cplx<float> o[2]) {
    reinterpret_cast<float4*>(v)[c] = make_float4(o[0].re, o[0].im, o[1].re, o[1].im);
  }
};
template <>
struct Chunk<double> {
  static constexpr int K = 1;
  __device__ __forceinline__ static void load(const double* v, size_t c, cplx<double> o[1]) {
    const double2 w = reinterpret_cast<const double2*>(v)[c];
    o[0] = {w.x, w.y};
  }
  __device__ __forceinline__ static void store(double* v, size_t c, const cplx<double> o[1]) {
    reinterpret_cast<double2*>(v)[c] = make_double2(o[0].re, o[0].im);
  }
};
// 16-bit inner vectors (FP16 or BF16 storage, FP32 arithmetic): four complex entries per 16-byte chunk,
// converted to FP32 on load and rounded to nearest on store.
template <>
struct Chunk<__half> {
  static constexpr int K = 4;
  __device__ __forceinline__ static void load(const __half* v, size_t c, cplx<float> o[4]) {
    const uint4 w = reinterpret_cast<const uint4*>(v)[c];
    const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u[k]));
      o[k] = {f.x, f.y};
    }
  }
  __device__ __forceinline__ static void store(__half* v, size_t c, const cplx<float> o[4]) {
    unsigned u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __half2 h = __floats2half2_rn(o[k].re, o[k].im);
      u[k] = *reinterpret_cast<const unsigned*>(&h);
    }
    reinterpret_cast<uint4*>(v)[c] = make_uint4(u[0], u[1], u[2], u[3]);
  }
};
template <>
struct Chunk<__nv_bfloat16> {
  static constexpr int K = 4;
  __device__ __forceinline__ static void load(const __nv_bfloat16* v, size_t c, cplx<float> o[4]) {
    const uint4 w = reinterpret_cast<const uint4*>(v)[c];
    const unsigned u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[k]));
      o[k] = {f.x, f.y};
    }
  }
  __device__ __forceinline__ static void store(__nv_bfloat16* v, size_t c, const cplx<float> o[4]) {
    unsigned u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(o[k].re, o[k].im);
      u[k] = *reinterpret_cast<const unsigned*>(&h);
    }
    reinterpret_cast<uint4*>(v)[c] = make_uint4(u[0], u[1], u[2], u[3]);
  }
};

// K complex entries starting at entry index e (a multiple of K), in as many chunks of X as needed.
template <typename X, int K>
__device__ __forceinline__ void load_k(const X* v, size_t e, cplx<typename Real<X>::acc> o[K]) {
  constexpr int KX = Chunk<X>::K;
  static_assert(K % KX == 0, "chunk sizes");
#pragma unroll
  for (int j = 0; j < K / KX; ++j) Chunk<X>::load(v, e / KX + j, o + j * KX);
}
template <typename X, int K>
__device__ __forceinline__ void store_k(X* v, size_t e, const cplx<typename Real<X>::acc> o[K]) {
  constexpr int KX = Chunk<X>::K;
#pragma unroll
  for (int j = 0; j < K / KX; ++j) Chunk<X>::store(v, e / KX + j, o + j * KX);
}

// End of a mixed-precision cycle: x (FP64) += scale * e (FP32 correction); e = 0.
__global__ void k_fold(double2* __restrict__ x, float* __restrict__ e, size_t n /* complex per rhs */,
                       const SolverState* st) {
  const int rh = blockIdx.y;
  const size_t off = (size_t)rh * n;
  const double s = st->scale[rh];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float2* ep = reinterpret_cast<float2*>(e) + off + i;
    const float2 ev = *ep;
    double2 xv = x[off + i];
    xv.x += s * (double)ev.x;
    xv.y += s * (double)ev.y;
    x[off + i] = xv;
    *ep = make_float2(0.f, 0.f);
  }
}

__global__ void k_new_cycle(SolverState* st) {
  st->done = 0;
  st->cycle_iter = 0;
}

// ------------------------------------------------------------------ fused update (one launch per iteration)
// Commit of one iteration by the last block at the fused update's grid barrier (one thread): tot[q] =
// |r_q|^2 after the r update. Forms beta = rr_new / rr, commits rr, per-rhs inner convergence, the
// iteration counts and the end-of-cycle flag.
__device__ __forceinline__ void commit_iteration(SolverState* st, const double* tot) {
  if (st->lanczos && !st->rhs_done[0] && st->lanczos_n < st->lanczos_cap) {
    st->lanczos[st->lanczos_n] = st->rr[0] / st->pAp[0];                      // alpha
    st->lanczos[st->lanczos_cap + st->lanczos_n] = tot[0] / st->rr[0];      // beta
    st->lanczos_n += 1;
  }
  bool all = true;
  for (int q = 0; q < st->nrhs; ++q) {
    st->rr_new[q] = tot[q];
    if (!st->rhs_done[q]) {
      if (!(st->pAp[q] > 0.0)) st->breakdown = 1;
      if (!isfinite(tot[q])) st->nonfinite = 1;
      st->beta[q] = tot[q] / st->rr[q];
      st->rr[q] = tot[q];
      const double s = st->scale[q];
      if (st->rr[q] * s * s <= st->tol2[q]) st->rhs_done[q] = 1;
    }
    all = all && st->rhs_done[q];
  }
  st->iter += 1;
  st->cycle_iter += 1;
  if (all || st->cycle_iter >= st->cycle_limit || st->breakdown || st->nonfinite) st->done = 1;
}

// The same commit by one full warp (warp 0 of the block that arrived last): lane q takes rhs q, q + 32,
// ...; lane 0 the counts, flags and the Lanczos record. Every value is loaded before the first store,
// so the commit costs about two L2 round trips instead of one per field.
__device__ __forceinline__ void commit_iteration_warp(SolverState* st, const double* tot) {
  const int lane = threadIdx.x & 31;
  const int nrhs = st->nrhs;
  int iter = 0, cyc = 0, lim = 0, brk = 0, nonf = 0, ln = 0, lcap = 0;
  double* lz = nullptr;
  if (lane == 0) {
    iter = st->iter;
    cyc = st->cycle_iter;
    lim = st->cycle_limit;
    brk = st->breakdown;
    nonf = st->nonfinite;
    lz = st->lanczos;
    ln = st->lanczos_n;
    lcap = st->lanczos_cap;
  }
  bool all = true, any_brk = false, any_nonf = false, lz_rec = false;
  double lz_alpha = 0.0, lz_beta = 0.0;
  for (int q0 = 0; q0 < nrhs; q0 += 32) {
    const int q = q0 + lane;
    bool done_q = true;
    if (q < nrhs) {
      const int rd = st->rhs_done[q];
      const double rr = st->rr[q], pap = st->pAp[q], sc = st->scale[q], tol2 = st->tol2[q], t = tot[q];
      if (q == 0 && !rd) {
        lz_rec = true;
        lz_alpha = rr / pap;
        lz_beta = t / rr;
      }
      st->rr_new[q] = t;
      done_q = rd != 0;
      if (!rd) {
        if (!(pap > 0.0)) any_brk = true;
        if (!isfinite(t)) any_nonf = true;
        st->beta[q] = t / rr;
        st->rr[q] = t;
        if (t * sc * sc <= tol2) {
          st->rhs_done[q] = 1;
          done_q = true;
        }
      }
    }
    all = __all_sync(0xffffffffu, done_q) && all;
    any_brk = __any_sync(0xffffffffu, any_brk);
    any_nonf = __any_sync(0xffffffffu, any_nonf);
  }
  if (lane == 0) {
    if (lz && lz_rec && ln < lcap) {
      lz[ln] = lz_alpha;
      lz[lcap + ln] = lz_beta;
      st->lanczos_n = ln + 1;
    }
    if (any_brk) st->breakdown = 1;
    if (any_nonf) st->nonfinite = 1;
    st->iter = iter + 1;
    st->cycle_iter = cyc + 1;
    if (all || cyc + 1 >= lim || brk || any_brk || nonf || any_nonf) st->done = 1;
  }
}

// The last block's part of the barrier: each warp sums the partials of some rhs ([rhs][gridDim.x x
// gridDim.y blocks], fixed order per lane, then a fixed shuffle tree), thread 0 commits the iteration.
__device__ __forceinline__ void finish_iteration(SolverState* st, const double* partials, int nblk, double* s_tot) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
  const int nrhs = st->nrhs;
  // whole warps only (a block of P * S threads may end in a partial warp)
  for (int q = warp; warp < nw && q < nrhs; q += nw) {
    const double t = warp_sum_partials(partials + (size_t)q * nblk, nblk);
    if (lane == 0) s_tot[q] = t;
  }
  __syncthreads();
  if (tid == 0) commit_iteration(st, s_tot);
}

// One CG iteration's vector updates in one launch on the blocked layout [rhs][cb][color] (grid: x
// chunks of a rhs, y = rhs; a cooperative launch of one wave):
//   phase 1: r -= alpha Ap (alpha = rr / pAp), rr_new = |r|^2 (per-chunk terms in the arithmetic
//            precision, FP64 over chunks);
//   barrier: one atomic per block; the last block to arrive releases the others at once, then every
//            block sums its rhs's partials (same order everywhere) into rr_new and beta, and the last
//            block also commits the iteration (counts, flags, Lanczos record);
//   phase 2: x += alpha p (X = double: the FP64 solution, X = float: the cycle's FP32 correction);
//            p = r + beta p.
// The first KEEP chunks of r a thread updates stay in registers for phase 2; further chunks are read
// again. Each thread handles its chunks in batches of KEEP whose loads are all issued before any store. Vector traffic: Ap, r read and r written, then p, x (and r beyond KEEP) read and p, x written:
// seven vector passes where an x/r update launch and a separate p update launch take nine.
template <typename S, typename X, int KEEP>
__global__ void __launch_bounds__(256, 4) k_cg_update(X* __restrict__ x, S* __restrict__ r, S* __restrict__ p,
                                                   const S* __restrict__ Ap, size_t n, SolverState* st,
                                                   double* partials, unsigned* bar) {
  using T = typename Real<S>::acc;
  using XT = typename Real<X>::acc;
  constexpr int K = Chunk<S>::K;
  __shared__ double red[32];
  __shared__ double s_tot[MAXR];
  __shared__ int s_last;
  if (st->done) return;  // uniform: only the last block at the barrier changes it
  const int rh = blockIdx.y;
  const size_t off = (size_t)rh * n;
  const double pap = st->pAp[rh];
  const bool frozen = st->rhs_done[rh] != 0;
  const bool active = !frozen && pap > 0.0 && isfinite(pap);
  const double rr_old = st->rr[rh];
  const double alpha = active ? rr_old / pap : 0.0;
  const T a = T(alpha);
  const XT ax = XT(sizeof(X) == 8 ? alpha * st->scale[rh] : alpha);
  const size_t stride = (size_t)gridDim.x * blockDim.x * K;
  const size_t i0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * K;
  const size_t nn = frozen ? 0 : n;  // a frozen rhs's vectors are not touched
  cplx<T> keep[KEEP][K];
  double v = 0.0;
  // phase 1 in batches of KEEP chunks: every load of a batch is issued before any store (r is read and
  // written, so a store would otherwise keep the next chunk's loads from being issued early)
  auto phase1 = [&](size_t ib, cplx<T>(&rv)[KEEP][K]) {
    cplx<T> av[KEEP][K];
#pragma unroll
    for (int j = 0; j < KEEP; ++j) {
      const size_t i = ib + j * stride;
      if (i < nn) {
        Chunk<S>::load(r, (off + i) / K, rv[j]);
        if (active) Chunk<S>::load(Ap, (off + i) / K, av[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < KEEP; ++j) {
      const size_t i = ib + j * stride;
      if (i < nn) {
        T t = T(0);
#pragma unroll
        for (int c = 0; c < K; ++c) {
          if (active) {
            rv[j][c].re = fma(-a, av[j][c].re, rv[j][c].re);
            rv[j][c].im = fma(-a, av[j][c].im, rv[j][c].im);
          }
          t += rv[j][c].re * rv[j][c].re + rv[j][c].im * rv[j][c].im;
        }
        if (active) Chunk<S>::store(r, (off + i) / K, rv[j]);
        v += (double)t;
      }
    }
  };
  phase1(i0, keep);  // the first batch stays in registers for phase 2
  for (size_t ib = i0 + KEEP * stride; ib < nn; ib += KEEP * stride) {
    cplx<T> rv[KEEP][K];
    phase1(ib, rv);
  }
  // phase 2 (x += alpha p, p = r + beta p), batch by batch: loads first, then the updates, then stores
  auto update_p_x = [&](double rr_new) {
    const T beta = T(rr_new / rr_old);
    auto phase2 = [&](size_t ib, const cplx<T>(&rv)[KEEP][K]) {
      cplx<T> pv[KEEP][K];
      cplx<XT> xv[KEEP][K];
#pragma unroll
      for (int j = 0; j < KEEP; ++j) {
        const size_t i = ib + j * stride;
        if (i < nn) {
          Chunk<S>::load(p, (off + i) / K, pv[j]);
          load_k<X, K>(x, off + i, xv[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < KEEP; ++j) {
        const size_t i = ib + j * stride;
        if (i < nn) {
#pragma unroll
          for (int c = 0; c < K; ++c) {
            xv[j][c].re = fma(ax, XT(pv[j][c].re), xv[j][c].re);
            xv[j][c].im = fma(ax, XT(pv[j][c].im), xv[j][c].im);
            pv[j][c].re = fma(beta, pv[j][c].re, rv[j][c].re);
            pv[j][c].im = fma(beta, pv[j][c].im, rv[j][c].im);
          }
          store_k<X, K>(x, off + i, xv[j]);
          Chunk<S>::store(p, (off + i) / K, pv[j]);
        }
      }
    };
    phase2(i0, keep);
    for (size_t ib = i0 + KEEP * stride; ib < nn; ib += KEEP * stride) {
      cplx<T> rv[KEEP][K];
#pragma unroll
      for (int j = 0; j < KEEP; ++j) {
        const size_t i = ib + j * stride;
        if (i < nn) Chunk<S>::load(r, (off + i) / K, rv[j]);
      }
      phase2(ib, rv);
    }
  };
  const double bs = block_sum_dyn(v, red);
  if (threadIdx.x == 0) partials[(size_t)rh * gridDim.x + blockIdx.x] = bs;
  unsigned gen;
  bool last;
  grid_arrive_release(bar, &gen, &last);
  if (!grid_wait64(bar, gen)) {
    if (threadIdx.x == 0) {
      st->timeout = 1;
      st->done = 1;
    }
    return;
  }
  // every block sums its rhs's partials itself (the same order in every block, so every block forms the
  // same beta); the block that arrived last also sums every rhs and commits the iteration
  if (threadIdx.x == 0) s_last = last ? 1 : 0;
  const double rr_new = block_sum_partials(partials + (size_t)rh * gridDim.x, gridDim.x, red);
  if (threadIdx.x == 0) s_tot[rh] = rr_new;
  if (active) update_p_x(rr_new);
  // after its own vectors (the flag is read back from shared memory so that nothing of this tail stays
  // in registers through phase 2): the other rhs's sums and the commit, read by the next launches only
  if (*(volatile int*)&s_last) {
    const int nrhs = st->nrhs;
    for (int q = 0; q < nrhs; ++q) {
      if (q == (int)blockIdx.y) continue;
      const double t = block_sum_partials(partials + (size_t)q * gridDim.x, gridDim.x, red);
      if (threadIdx.x == 0) s_tot[q] = t;
    }
    __syncthreads();
    if (threadIdx.x < 32) commit_iteration_warp(st, s_tot);
  }
}

// ------------------------------------------------------------------ rhs-interleaved inner vectors
// Mixed-precision multi-RHS solves with an even number N of rhs keep their FP32 inner vectors in the
// rhs-interleaved layout [cb][color][rhs] that the interleaved Dslash reads. Every 16-byte word holds
// one colour of rhs 2q and 2q+1 at one site: word w = (3 cb + colour) P + q with P = N / 2. A block of
// P * S threads (S a power of two) and a grid stride that is a multiple of P keep q = tid % P fixed
// for every word a thread touches, so each thread carries the scalars of one rhs pair.
__device__ __forceinline__ void wload(const float* base, size_t w, cplx<float> (&v)[2]) {
  const float4 a = reinterpret_cast<const float4*>(base)[w];
  v[0] = {a.x, a.y};
  v[1] = {a.z, a.w};
}
__device__ __forceinline__ void wstore(float* base, size_t w, const cplx<float> (&v)[2]) {
  reinterpret_cast<float4*>(base)[w] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
}

// Sum of v[0..1] over the S slots (tid / P) of the block for each rhs pair q = tid % P (a tree over S);
// the threads tid < P get the totals of pair tid.
__device__ __forceinline__ void il_block_sum(double (&v)[2], int P, double* red /* [2][blockDim] */) {
  const int S = blockDim.x / P, q = threadIdx.x % P, y = threadIdx.x / P, nt = P * S;
  red[y * P + q] = v[0];
  red[nt + y * P + q] = v[1];
  __syncthreads();
  for (int h = S >> 1; h > 0; h >>= 1) {
    if (y < h) {
      red[y * P + q] += red[(y + h) * P + q];
      red[nt + y * P + q] += red[nt + (y + h) * P + q];
    }
    __syncthreads();
  }
  v[0] = red[q];
  v[1] = red[nt + q];
}

// The fused update (as k_cg_update) on interleaved FP32 vectors; e: the cycle's FP32 correction,
// interleaved as well. nw: 16-byte words per vector set (3 * half * P). Phase 2 reads r again (the N
// vectors of a thread's words do not fit in registers).
__global__ void __launch_bounds__(256) k_cg_update_il(float* __restrict__ e, float* __restrict__ r,
                                                      float* __restrict__ p, const float* __restrict__ Ap,
                                                      size_t nw, int P, SolverState* st, double* partials,
                                                      unsigned* bar) {
  __shared__ double red[512];
  __shared__ double s_tot[MAXR];
  if (st->done) return;  // uniform: only the last block at the barrier changes it
  const int q = threadIdx.x % P;
  bool active[2], frozen[2];
  float a[2];
  for (int k = 0; k < 2; ++k) {
    const int rh = 2 * q + k;
    const double pap = st->pAp[rh];
    frozen[k] = st->rhs_done[rh] != 0;
    active[k] = !frozen[k] && pap > 0.0 && isfinite(pap);
    a[k] = active[k] ? float(st->rr[rh] / pap) : 0.f;
  }
  const bool any = !frozen[0] || !frozen[1];
  const size_t w0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  constexpr int BW = 4;  // words per batch: all loads of a batch are issued before its stores
  double v[2] = {0.0, 0.0};
  for (size_t wb = any ? w0 : nw; wb < nw; wb += BW * stride) {
    cplx<float> rv[BW][2], av[BW][2];
#pragma unroll
    for (int j = 0; j < BW; ++j) {
      const size_t w = wb + j * stride;
      if (w < nw) {
        wload(r, w, rv[j]);
        if (active[0] || active[1]) wload(Ap, w, av[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < BW; ++j) {
      const size_t w = wb + j * stride;
      if (w < nw) {
        if (active[0] || active[1]) {
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            rv[j][k].re = fma(-a[k], av[j][k].re, rv[j][k].re);
            rv[j][k].im = fma(-a[k], av[j][k].im, rv[j][k].im);
          }
          wstore(r, w, rv[j]);
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) v[k] += (double)(rv[j][k].re * rv[j][k].re + rv[j][k].im * rv[j][k].im);
      }
    }
  }
  il_block_sum(v, P, red);
  if (threadIdx.x < P) {
    partials[(size_t)(2 * q) * gridDim.x + blockIdx.x] = v[0];
    partials[(size_t)(2 * q + 1) * gridDim.x + blockIdx.x] = v[1];
  }
  unsigned gen;
  if (grid_arrive(bar, &gen)) {
    finish_iteration(st, partials, gridDim.x, s_tot);
    grid_release(bar);
  } else if (!grid_wait(bar, gen)) {
    if (threadIdx.x == 0) {
      st->timeout = 1;
      st->done = 1;
    }
    return;
  }
  if (!active[0] && !active[1]) return;
  float beta[2];
  for (int k = 0; k < 2; ++k) beta[k] = active[k] ? float(__ldcg(&st->beta[2 * q + k])) : 0.f;
  for (size_t wb = w0; wb < nw; wb += BW * stride) {
    cplx<float> rv[BW][2], pv[BW][2], ev[BW][2];
#pragma unroll
    for (int j = 0; j < BW; ++j) {
      const size_t w = wb + j * stride;
      if (w < nw) {
        wload(r, w, rv[j]);
        wload(p, w, pv[j]);
        wload(e, w, ev[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < BW; ++j) {
      const size_t w = wb + j * stride;
      if (w >= nw) continue;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (!active[k]) continue;  // a frozen rhs keeps its p and e
        ev[j][k].re = fma(a[k], pv[j][k].re, ev[j][k].re);
        ev[j][k].im = fma(a[k], pv[j][k].im, ev[j][k].im);
        pv[j][k].re = fma(beta[k], pv[j][k].re, rv[j][k].re);
        pv[j][k].im = fma(beta[k], pv[j][k].im, rv[j][k].im);
      }
      wstore(e, w, ev[j]);
      wstore(p, w, pv[j]);
    }
  }
}

// Reliable update on interleaved FP32 vectors: for each unverified rhs, r_lo = p = r_hi / s from the
// blocked FP64 residual r_hi ([rhs][cb][color]); then (last block) the bookkeeping of k_reliable.
__global__ void k_reliable_il(const double2* __restrict__ r_hi, float* __restrict__ r_lo, float* __restrict__ p,
                              size_t nw, int P, SolverState* st, unsigned* counter) {
  const int q = threadIdx.x % P;
  const size_t n = nw / P;  // complex entries per rhs (3 * half)
  double inv[2];
  bool upd[2];
  for (int k = 0; k < 2; ++k) {
    const int rh = 2 * q + k;
    const double s_new = sqrt(st->rr_true[rh] / (double)n);
    upd[k] = !(st->rr_true[rh] <= st->tol2[rh]) && s_new > 0.0;
    inv[k] = upd[k] ? 1.0 / s_new : 0.0;
  }
  if (upd[0] || upd[1]) {
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < nw; w += (size_t)gridDim.x * blockDim.x) {
      const size_t entry = w / P;  // 3 cb + colour
      cplx<float> rv[2], pv[2];
      wload(r_lo, w, rv);
      wload(p, w, pv);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (!upd[k]) continue;
        const double2 h = r_hi[(size_t)(2 * q + k) * n + entry];
        rv[k] = {float(h.x * inv[k]), float(h.y * inv[k])};
        pv[k] = rv[k];
      }
      wstore(r_lo, w, rv);
      wstore(p, w, pv);
    }
  }
  if (last_block_done(counter) && threadIdx.x == 0) reliable_commit(st, n);
}

// End of a mixed-precision cycle on interleaved corrections: x (blocked FP64) += scale * e; e = 0.
__global__ void k_fold_il(double2* __restrict__ x, float* __restrict__ e, size_t nw, int P, const SolverState* st) {
  const int q = threadIdx.x % P;
  const size_t n = nw / P;
  const double s[2] = {st->scale[2 * q], st->scale[2 * q + 1]};
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < nw; w += (size_t)gridDim.x * blockDim.x) {
    const size_t entry = w / P;
    cplx<float> ev[2];
    wload(e, w, ev);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      double2* dst = x + (size_t)(2 * q + k) * n + entry;
      double2 xv = *dst;
      xv.x += s[k] * (double)ev[k].re;
      xv.y += s[k] * (double)ev[k].im;
      *dst = xv;
    }
    const cplx<float> z[2] = {{0.f, 0.f}, {0.f, 0.f}};
    wstore(e, w, z);
  }
}

// ------------------------------------------------------------------ host driver
struct CgBuffers {
  double2 *x, *b, *r_hi, *Ax, *t64;
  size_t b_stride;          // complex entries between sources (0: one source for every rhs)
  std::vector<double> a;    // per-rhs diagonal 4m^2 + sigma_r
  void *r, *p, *Ap, *t;  // inner vectors (S = double or float)
  void* e;               // mixed precision: FP32 correction of the current cycle (else == x)
  SolverState* st;
  double* partials;
  int rp = HISQ_F64;     // operator precision of the true residual: HISQ_F64 or HISQ_DF64
  unsigned* rowc;        // per-rhs block counters of the row reductions [MAXR]
  bool il = false;       // inner vectors (r, p, Ap, t, e) in the rhs-interleaved layout [cb][color][rhs]
  int P = 0;             // il: rhs pairs per site (nrhs / 2)
  int il_block = 0;      // il: threads per block of the interleaved BLAS kernels (P x a power of two)
  dim3 upd_grid;         // the fused update's cooperative grid (one wave)
  int upd_block = 256;
};

// Cooperative launch (every block resident at once: the fused update meets at a grid barrier).
template <typename... Exp, typename... Act>
static cudaError_t launch_cooperative(void (*kernel)(Exp...), dim3 grid, int block, cudaStream_t stream,
                                      Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Act>(args)...);
}

// The fused update kernel for the buffers' layout and inner type.
template <typename S>
static const void* update_kernel(const CgBuffers& B) {
  if (B.il) return (const void*)k_cg_update_il;
  if constexpr (sizeof(S) == 8) return (const void*)k_cg_update<double, double, 2>;
  if constexpr (sizeof(S) == 2) return (const void*)k_cg_update<S, float, 1>;  // 4 entries a chunk
  return (const void*)k_cg_update<float, float, 2>;
}

// One wave of the fused update: as many blocks as are resident together, at most one per unit of work.
template <typename S>
static int plan_update(hisq_ctx* ctx, CgBuffers& B, int nrhs) {
  int per_sm = 0;
  B.upd_block = B.il ? B.il_block : 256;
  HISQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, update_kernel<S>(B), B.upd_block, 0));
  if (per_sm < 1) return set_error(HISQ_ECUDA, "fused CG update cannot be resident");
  const size_t wave = (size_t)ctx->num_sms * per_sm;
  if (B.il) {
    const size_t words = (size_t)ctx->g.half * 3 * B.P;
    size_t gx = (words + B.il_block - 1) / B.il_block;
    B.upd_grid = dim3((unsigned)(gx < wave ? gx : wave), 1);
  } else {
    const size_t chunks = (size_t)ctx->g.half * 3 / Chunk<S>::K;
    size_t gx = (chunks + B.upd_block - 1) / B.upd_block;
    const size_t cap = wave / (size_t)nrhs;
    if (cap < 1) return set_error(HISQ_EINVAL, "%d rhs exceed one wave of the fused CG update", nrhs);
    B.upd_grid = dim3((unsigned)(gx < cap ? gx : cap), nrhs);
  }
  return HISQ_OK;
}

static dim3 blas_grid(const hisq_ctx* ctx, int nrhs, size_t units, int per_sm = 8) {
  size_t gx = (units + 255) / 256;
  const size_t cap = (size_t)ctx->num_sms * per_sm;  // one wave of 256-thread blocks (grid-stride beyond)
  if (gx > cap) gx = cap;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, nrhs);
}
static dim3 blas_grid(const hisq_ctx* ctx, int nrhs) { return blas_grid(ctx, nrhs, (size_t)ctx->g.half); }

// r_hi = b - A x with the reliable-update operator (FP64, or double-float); rr_true (and bb with init).
static int true_residual(hisq_ctx* ctx, const CgBuffers& B, int nrhs, int init) {
  const size_t n = (size_t)ctx->g.half * 3;
  DslashCall c1;
  c1.out_parity = 1;
  c1.out = B.t64;
  c1.in = B.x;
  c1.nrhs = nrhs;
  c1.rhs_stride = ctx->g.half;
  int rc = dslash_launch(ctx, B.rp, HISQ_F64, c1);
  if (rc != HISQ_OK) return rc;
  DslashCall c2 = c1;
  c2.out_parity = 0;
  c2.out = B.Ax;
  c2.in = B.t64;
  c2.y = B.x;
  c2.a_rhs = B.a.data();
  c2.epi = EPI_AXPY;
  if ((rc = dslash_launch(ctx, B.rp, HISQ_F64, c2)) != HISQ_OK) return rc;
  k_residual<<<blas_grid(ctx, nrhs), 256, 0, ctx->stream>>>(B.b, B.b_stride, B.Ax, B.r_hi, n, B.st, B.partials,
                                                            partial_stride(ctx), ctx->d_counters + 1, init);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  return HISQ_OK;
}

// Grid of the interleaved BLAS kernels: one thread per 16-byte word, at most one wave of 8 blocks per SM
// (the grid stride stays a multiple of P, as every block is).
static dim3 il_grid(const hisq_ctx* ctx, const CgBuffers& B) {
  const size_t words = (size_t)ctx->g.half * 3 * B.P;
  size_t gx = (words + B.il_block - 1) / B.il_block;
  const size_t cap = (size_t)ctx->num_sms * 8;
  return dim3((unsigned)(gx < cap ? gx : cap));
}

template <typename S>
static int reliable(hisq_ctx* ctx, const CgBuffers& B, int nrhs, int first) {
  const size_t n = (size_t)ctx->g.half * 3;
  if (B.il) {
    k_reliable_il<<<il_grid(ctx, B), B.il_block, 0, ctx->stream>>>(B.r_hi, (float*)B.r, (float*)B.p,
                                                                   n * B.P, B.P, B.st, ctx->d_counters + 2);
    HISQ_CUDA(cudaGetLastError());
    note_launch(ctx);
    return HISQ_OK;
  }
  k_reliable<S><<<blas_grid(ctx, nrhs), 256, 0, ctx->stream>>>(B.r_hi, (S*)B.r, (S*)B.p, n, B.st, first,
                                                               ctx->d_counters + 2);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  return HISQ_OK;
}

// One inner iteration (inner link precision lp, spinor type S). Mixed precision accumulates
// the cycle's correction e in FP32; k_fold adds it to the FP64 x before each reliable update.
template <typename S>
static int iteration(hisq_ctx* ctx, const CgBuffers& B, int lp, int nrhs) {
  const int sp = Real<S>::prec;
  const size_t n = (size_t)ctx->g.half * 3;
  DslashCall c1;
  c1.out_parity = 1;
  c1.out = B.t;
  c1.in = B.p;
  c1.nrhs = nrhs;
  c1.rhs_stride = ctx->g.half;
  c1.skip = &B.st->done;
  c1.interleaved = B.il;
  int rc = dslash_launch(ctx, lp, sp, c1);
  if (rc != HISQ_OK) return rc;
  DslashCall c2 = c1;
  c2.out_parity = 0;
  c2.out = B.Ap;
  c2.in = B.t;
  c2.y = B.p;
  c2.a_rhs = B.a.data();
  c2.epi = EPI_AXPY;
  c2.partials = B.partials + 2 * MAXR * partial_stride(ctx);
  c2.dot_out = B.st->pAp;
  c2.counter = ctx->d_counters + 3;
  if ((rc = dslash_launch(ctx, lp, sp, c2)) != HISQ_OK) return rc;
  // the vector updates of the iteration: one cooperative launch meeting at a grid barrier
  unsigned* bar = ctx->d_counters + 30;
  cudaError_t e;
  if (B.il)
    e = launch_cooperative(k_cg_update_il, B.upd_grid, B.upd_block, ctx->stream, (float*)B.e, (float*)B.r,
                           (float*)B.p, (const float*)B.Ap, n * B.P, B.P, B.st, B.partials, bar);
  else if constexpr (sizeof(S) == 8)
    e = launch_cooperative(k_cg_update<double, double, 2>, B.upd_grid, B.upd_block, ctx->stream, (double*)B.x,
                           (double*)B.r, (double*)B.p, (const double*)B.Ap, n, B.st, B.partials, bar);
  else if constexpr (sizeof(S) == 2)
    e = launch_cooperative(k_cg_update<S, float, 1>, B.upd_grid, B.upd_block, ctx->stream, (float*)B.e, (S*)B.r,
                           (S*)B.p, (const S*)B.Ap, n, B.st, B.partials, bar);
  else
    e = launch_cooperative(k_cg_update<float, float, 2>, B.upd_grid, B.upd_block, ctx->stream, (float*)B.e,
                           (float*)B.r, (float*)B.p, (const float*)B.Ap, n, B.st, B.partials, bar);
  HISQ_CUDA(e);
  note_launch(ctx);
  return HISQ_OK;
}

// ------------------------------------------------------------------ Lanczos estimate of the spectrum
// CG's coefficients define the Lanczos tridiagonal matrix T of A on the Krylov space of the source:
// T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_k,k+1 = sqrt(beta_k)/alpha_k. Its extreme eigenvalues
// approach A's from inside as the iteration proceeds. They are found by bisection on the Sturm count
// (the number of negative pivots of T - x I is the number of eigenvalues below x).
static int sturm_count(const std::vector<double>& d, const std::vector<double>& e2, double x) {
  int neg = 0;
  double q = 1.0;
  for (size_t k = 0; k < d.size(); ++k) {
    q = d[k] - x - (k > 0 ? e2[k - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;  // a zero pivot counts as negative: x sits on an eigenvalue
    if (q < 0.0) ++neg;
  }
  return neg;
}

int lanczos_extremes(const double* alpha, const double* beta, int n, double* lmin, double* lmax) {
  // the longest run of coefficients between restarts (alpha = 0)
  int best0 = 0, bestn = 0;
  for (int k = 0; k < n;) {
    int j = k;
    while (j < n && alpha[j] > 0.0 && std::isfinite(alpha[j]) && beta[j] >= 0.0) ++j;
    if (j - k > bestn) {
      best0 = k;
      bestn = j - k;
    }
    k = j + 1;
  }
  if (bestn < 1) return set_error(HISQ_EINVAL, "no Lanczos coefficients");
  std::vector<double> d(bestn), e2(bestn > 1 ? bestn - 1 : 1, 0.0);
  double lo = 1e300, hi = -1e300;
  for (int k = 0; k < bestn; ++k) {
    const double* a = alpha + best0;
    const double* b = beta + best0;
    d[k] = 1.0 / a[k] + (k > 0 ? b[k - 1] / a[k - 1] : 0.0);
    if (k + 1 < bestn) e2[k] = b[k] / (a[k] * a[k]);
  }
  for (int k = 0; k < bestn; ++k) {  // Gershgorin bounds
    const double r = (k > 0 ? sqrt(e2[k - 1]) : 0.0) + (k + 1 < bestn ? sqrt(e2[k]) : 0.0);
    lo = fmin(lo, d[k] - r);
    hi = fmax(hi, d[k] + r);
  }
  auto bisect = [&](int target) {  // the smallest x with count(x) > target
    double a = lo, b = hi;
    for (int it = 0; it < 200 && b - a > 1e-15 * fmax(fabs(a), fabs(b)); ++it) {
      const double m = 0.5 * (a + b);
      if (sturm_count(d, e2, m) > target) b = m;
      else a = m;
    }
    return 0.5 * (a + b);
  };
  *lmin = bisect(0);
  *lmax = bisect(bestn - 1);
  return HISQ_OK;
}

// CG for nrhs systems (A + sigma_r) x_r = b_r at once. x: device FP64 [nrhs][half][3]
// (initial guess in, solution out); b: device FP64 sources with b_stride complex entries
// between consecutive sources (0: one source for all rhs). sigma, tol: host arrays [nrhs].
template <typename S>
static int run_cg(hisq_ctx* ctx, double2* x, const double2* b, size_t b_stride, int nrhs, double mass,
                  const double* sigma, const double* tol, int maxiter, const hisq_solver_opts& o,
                  hisq_solver_stats* stats) {
  auto t_start = std::chrono::steady_clock::now();
  const int lp = o.inner_prec;
  // FP32 or 16-bit inner vectors: mixed precision (FP64 and double-float CG are plain)
  const bool mixed = sizeof(S) <= 4;
  const int sp = Real<S>::prec;
  const size_t n = (size_t)ctx->g.half * 3;
  const size_t vb64 = (size_t)nrhs * n * sizeof(double2);
  const size_t vbS = (size_t)nrhs * n * 2 * sizeof(S);
  CgBuffers B;
  B.rp = o.reliable_prec;
  B.x = x;
  B.b = const_cast<double2*>(b);
  B.b_stride = b_stride;
  B.r_hi = (double2*)workspace(ctx, "cg_rhi", vb64);
  B.Ax = (double2*)workspace(ctx, "cg_Ax", vb64);
  B.t64 = (double2*)workspace(ctx, "cg_t64", vb64);
  B.r = workspace(ctx, "cg_r", vbS);
  B.p = workspace(ctx, "cg_p", vbS);
  B.Ap = workspace(ctx, "cg_Ap", vbS);
  B.t = workspace(ctx, "cg_t", vbS);
  B.st = (SolverState*)workspace(ctx, "cg_state", sizeof(SolverState));
  B.partials = (double*)workspace(ctx, "cg_partials", 3 * MAXR * partial_stride(ctx) * sizeof(double));
  B.rowc = (unsigned*)workspace(ctx, "cg_rowc", MAXR * sizeof(unsigned));
  B.e = mixed ? workspace(ctx, "cg_e", (size_t)nrhs * n * 2 * sizeof(float)) : (void*)x;
  SolverState* hst = (SolverState*)ctx->pinned;
  if (!B.r_hi || !B.Ax || !B.t64 || !B.r || !B.p || !B.Ap || !B.t || !B.st || !B.partials || !B.e || !B.rowc)
    return set_error(HISQ_ENOMEM, "solver workspace");
  // on request (vector_layout 1), mixed precision with an even number of rhs keeps its inner vectors
  // interleaved per site, so the Dslash reads each neighbour's nrhs vectors as one block
  B.il = std::is_same<S, float>::value && nrhs >= 2 && nrhs % 2 == 0 && o.vector_layout == 1;
  if (B.il) {
    B.P = nrhs / 2;
    int spb = 1;
    while (B.P * spb * 2 <= 256) spb *= 2;
    B.il_block = B.P * spb;
  }
  int prc = plan_update<S>(ctx, B, nrhs);
  if (prc != HISQ_OK) return prc;
  HISQ_CUDA(cudaMemsetAsync(B.rowc, 0, MAXR * sizeof(unsigned), ctx->stream));
  if (mixed) HISQ_CUDA(cudaMemsetAsync(B.e, 0, (size_t)nrhs * n * 2 * sizeof(float), ctx->stream));
  auto fold = [&]() -> int {
    if (!mixed) return HISQ_OK;
    if (B.il) {
      k_fold_il<<<il_grid(ctx, B), B.il_block, 0, ctx->stream>>>(B.x, (float*)B.e, n * B.P, B.P, B.st);
      HISQ_CUDA(cudaGetLastError());
      note_launch(ctx);
      return HISQ_OK;
    }
    k_fold<<<blas_grid(ctx, nrhs, n), 256, 0, ctx->stream>>>(B.x, (float*)B.e, n, B.st);
    HISQ_CUDA(cudaGetLastError());
    note_launch(ctx);
    return HISQ_OK;
  };
  B.a.resize(nrhs);
  for (int q = 0; q < nrhs; ++q) B.a[q] = 4.0 * mass * mass + (sigma ? sigma[q] : 0.0);
  long long dcalls = 0;
  double dbytes = 0.0;

  constexpr int LANCZOS_CAP = 4096;
  double* lanczos = (double*)workspace(ctx, "cg_lanczos", 2 * LANCZOS_CAP * sizeof(double));
  if (!lanczos) return set_error(HISQ_ENOMEM, "solver workspace");
  memset(hst, 0, sizeof(SolverState));
  hst->lanczos = lanczos;
  hst->lanczos_cap = LANCZOS_CAP;
  hst->nrhs = nrhs;
  hst->cycle_limit = mixed ? o.reliable_period : o.poll_every;
  for (int q = 0; q < nrhs; ++q) hst->scale[q] = 1.0;
  HISQ_CUDA(cudaMemcpyAsync(B.st, hst, sizeof(SolverState), cudaMemcpyHostToDevice, ctx->stream));
  // a zero initial guess (the usual start) needs no A x: its residual is b
  double* xn = (double*)ctx->pinned + 4096;
  k_xnorm<<<blas_grid(ctx, nrhs, n), 256, 0, ctx->stream>>>(x, n, nrhs, B.partials, partial_stride(ctx),
                                                             ctx->d_counters + 10, (double*)B.Ax);
  HISQ_CUDA(cudaGetLastError());
  HISQ_CUDA(cudaMemcpyAsync(xn, B.Ax, nrhs * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  note_launch(ctx);
  bool x_zero = true;
  for (int q = 0; q < nrhs; ++q) x_zero = x_zero && xn[q] == 0.0;
  int rc;
  if (x_zero) {
    k_residual_zero<<<blas_grid(ctx, nrhs), 256, 0, ctx->stream>>>(B.b, B.b_stride, B.r_hi, n, B.st, B.partials,
                                                                    partial_stride(ctx), ctx->d_counters + 1);
    HISQ_CUDA(cudaGetLastError());
    note_launch(ctx);
  } else {
    if ((rc = true_residual(ctx, B, nrhs, 1)) != HISQ_OK) return rc;
    dcalls += 2;
    dbytes += 2 * dslash_bytes(ctx, B.rp, HISQ_F64, nrhs);
  }
  HISQ_CUDA(cudaMemcpyAsync(hst, B.st, sizeof(SolverState), cudaMemcpyDeviceToHost, ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int q = 0; q < nrhs; ++q) {
    if (!isfinite(hst->bb[q]) || !isfinite(hst->rr_true[q]))
      return set_error(HISQ_ENONFINITE, "non-finite source or initial guess (rhs %d)", q);
    hst->tol2[q] = tol[q] * tol[q] * hst->bb[q];
    if (hst->bb[q] == 0.0) {
      // a zero source has the exact solution x = 0 (its relative residual is not defined)
      HISQ_CUDA(cudaMemsetAsync(x + (size_t)q * n, 0, n * sizeof(double2), ctx->stream));
      hst->rr_true[q] = 0.0;
    }
  }
  HISQ_CUDA(cudaMemcpyAsync(B.st, hst, sizeof(SolverState), cudaMemcpyHostToDevice, ctx->stream));
  if ((rc = reliable<S>(ctx, B, nrhs, 1)) != HISQ_OK) return rc;

  const int cycle = hst->cycle_limit;
  cudaGraphExec_t exec = nullptr;
  long long graph_nodes = 0;
  if (o.use_graph) {
    // a cycle's graph depends on the buffers, shapes and per-rhs coefficients it was captured with
    std::string key = "cg/" + std::to_string(sizeof(S)) + "/" + std::to_string(lp) + "/" + std::to_string(nrhs) +
                      (B.il ? "/il" : "/bl") +
                      "/" + std::to_string(cycle);
    char buf[64];
    for (const void* ptr : {(const void*)B.r, (const void*)B.p, (const void*)B.Ap, (const void*)B.t,
                            (const void*)B.e, (const void*)B.st, (const void*)B.partials, (const void*)B.rowc}) {
      snprintf(buf, sizeof buf, "/%p", ptr);
      key += buf;
    }
    for (double a : B.a) {
      snprintf(buf, sizeof buf, "/%a", a);
      key += buf;
    }
    auto cached = ctx->graphs.find(key);
    if (cached != ctx->graphs.end()) {
      exec = cached->second.first;
      graph_nodes = cached->second.second;
    } else {
      // tune the inner Dslash launches outside the capture (they are idempotent)
      DslashCall c1;
      c1.out_parity = 1;
      c1.out = B.t;
      c1.in = B.p;
      c1.nrhs = nrhs;
      c1.rhs_stride = ctx->g.half;
      c1.interleaved = B.il;
      if ((rc = dslash_launch(ctx, lp, sp, c1)) != HISQ_OK) return rc;
      DslashCall c2 = c1;
      c2.out_parity = 0;
      c2.out = B.Ap;
      c2.in = B.t;
      c2.y = B.p;
      c2.a_rhs = B.a.data();
      c2.epi = EPI_AXPY;
      c2.partials = B.partials + 2 * MAXR * partial_stride(ctx);
      c2.dot_out = B.st->pAp;
      c2.counter = ctx->d_counters + 3;
      if ((rc = dslash_launch(ctx, lp, sp, c2)) != HISQ_OK) return rc;

      TraceRange trace("cg graph capture");
      cudaGraph_t graph;
      HISQ_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      ctx->capturing = true;
      int crc = HISQ_OK;
      for (int i = 0; i < cycle && crc == HISQ_OK; ++i) crc = iteration<S>(ctx, B, lp, nrhs);
      ctx->capturing = false;
      cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
      if (crc != HISQ_OK) return crc;
      HISQ_CUDA(ce);
      size_t nodes = 0;
      cudaGraphGetNodes(graph, nullptr, &nodes);
      graph_nodes = (long long)nodes;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      HISQ_CUDA(ce);
      if (ctx->graphs.size() >= 32) release_graphs(ctx);  // bound the cache
      ctx->graphs[key] = {exec, graph_nodes};
    }
  }
  auto run_cycle = [&]() -> int {
    if (exec) {
      HISQ_CUDA(cudaGraphLaunch(exec, ctx->stream));
      ctx->launches += graph_nodes;
      return HISQ_OK;
    }
    for (int i = 0; i < cycle; ++i) {
      int r2 = iteration<S>(ctx, B, lp, nrhs);
      if (r2 != HISQ_OK) return r2;
    }
    return HISQ_OK;
  };

  int status = HISQ_OK;
  int reliable_updates = 0;
  HISQ_CUDA(cudaMemcpyAsync(hst, B.st, sizeof(SolverState), cudaMemcpyDeviceToHost, ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  bool converged = hst->done != 0;
  bool verified = true;  // rr_true reflects the current x
  int last_iter = 0;
  while (!converged) {
    if (hst->iter >= maxiter) {
      status = HISQ_ENOCONV;
      break;
    }
    if ((rc = run_cycle()) != HISQ_OK) {
      status = rc;
      break;
    }
    verified = false;
    HISQ_CUDA(cudaMemcpyAsync(hst, B.st, sizeof(SolverState), cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    const int done_iters = hst->iter - last_iter;
    last_iter = hst->iter;
    dcalls += 2LL * done_iters;
    dbytes += 2.0 * done_iters * dslash_bytes(ctx, lp, sp, nrhs);
    if (hst->timeout) {
      status = set_error(HISQ_ETIMEOUT, "a grid-barrier wait of the CG update ran out at iteration %d", hst->iter);
      break;
    }
    if (hst->nonfinite) {
      status = set_error(HISQ_ENONFINITE, "non-finite residual at iteration %d", hst->iter);
      break;
    }
    if (hst->breakdown) {
      status = set_error(HISQ_EBREAKDOWN, "<p, A p> <= 0 at iteration %d", hst->iter);
      break;
    }
    bool all_inner = true;
    for (int q = 0; q < nrhs; ++q) all_inner = all_inner && hst->rhs_done[q];
    if (mixed || all_inner) {
      TraceRange trace("reliable update");
      if ((rc = fold()) != HISQ_OK) return rc;
      if ((rc = true_residual(ctx, B, nrhs, 0)) != HISQ_OK) return rc;
      if ((rc = reliable<S>(ctx, B, nrhs, 0)) != HISQ_OK) return rc;
      dcalls += 2;
      dbytes += 2 * dslash_bytes(ctx, B.rp, HISQ_F64, nrhs);
      ++reliable_updates;
      verified = true;
      HISQ_CUDA(cudaMemcpyAsync(hst, B.st, sizeof(SolverState), cudaMemcpyDeviceToHost, ctx->stream));
      HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
      converged = true;
      for (int q = 0; q < nrhs; ++q) converged = converged && hst->rhs_conv[q];
    } else {
      k_new_cycle<<<1, 1, 0, ctx->stream>>>(B.st);
      HISQ_CUDA(cudaGetLastError());
      note_launch(ctx);
    }
  }
  if (!verified) {
    // the iterate changed since the last true residual: recompute it for the report
    if ((rc = fold()) != HISQ_OK) return rc;
    if ((rc = true_residual(ctx, B, nrhs, 0)) != HISQ_OK) return rc;
    HISQ_CUDA(cudaMemcpyAsync(hst, B.st, sizeof(SolverState), cudaMemcpyDeviceToHost, ctx->stream));
  }
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  double worst = 0.0;
  for (int q = 0; q < nrhs; ++q) {
    double rel = hst->bb[q] > 0 ? sqrt(hst->rr_true[q] / hst->bb[q]) : sqrt(hst->rr_true[q]);
    if (rel > worst) worst = rel;
    if (stats && q < 64) stats->shift_residual[q] = rel;
  }
  if (stats) {
    stats->iters += hst->iter;
    stats->reliable_updates += reliable_updates;
    stats->converged = converged && status == HISQ_OK;
    stats->true_rel_residual = worst;
    stats->seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    stats->dslash_bytes += dbytes;
    stats->dslash_calls += dcalls;
    // the estimate of A's extreme eigenvalues from rhs 0's Lanczos coefficients
    const int nl = hst->lanczos_n;
    stats->lanczos_steps = nl;
    if (nl > 0) {
      std::vector<double> ab(2 * (size_t)LANCZOS_CAP);
      HISQ_CUDA(cudaMemcpy(ab.data(), lanczos, ab.size() * sizeof(double), cudaMemcpyDeviceToHost));
      if (lanczos_extremes(ab.data(), ab.data() + LANCZOS_CAP, nl, &stats->lambda_min, &stats->lambda_max) != HISQ_OK)
        stats->lambda_min = stats->lambda_max = 0.0;
    }
  }
  if (status == HISQ_ENOCONV)
    return set_error(HISQ_ENOCONV, "no convergence in %d iterations (true residual %.3e)", hst->iter, worst);
  return status;
}

// ------------------------------------------------------------------ multi-shift CG
// Shifted systems (A + sigma_k) x_k = b share the Krylov space of the base system (smallest
// shift): r_k = zeta_k r. Per base iteration j (Jegerlehner's recurrences, hep-lat/9612014):
//   zeta_k' = zeta_k zeta_k^old alpha_old / (alpha beta_old (zeta_k^old - zeta_k)
//                                            + zeta_k^old alpha_old (1 + (sigma_k - sigma_0) alpha))
//   alpha_k = alpha zeta_k'/zeta_k,  x_k += alpha_k p_k,
//   beta_k  = beta (zeta_k'/zeta_k)^2,  p_k = zeta_k' r + beta_k p_k.
struct MsState {
  double sigma[MAXR], zeta[MAXR], zeta_old[MAXR], zeta_new[MAXR], alpha_k[MAXR], beta_k[MAXR], tol2[MAXR];
  int active[MAXR], conv_iter[MAXR];
  double rr, rr_new, pAp, bb, alpha, alpha_old, beta_old, scale;
  int base, nshift, iter, done, cycle_iter, cycle_limit, breakdown, nonfinite;
};

// r -= alpha Ap (alpha = rr / pAp), rr_new = |r|^2; last block: every shift's recurrence scalars.
template <typename S>
__global__ void k_ms_rupdate(S* __restrict__ r, const S* __restrict__ Ap, size_t n, MsState* st, double* partials,
                             size_t pstride, unsigned* counter) {
  if (st->done) return;
  using T = typename Real<S>::acc;
  constexpr int K = Chunk<S>::K;
  const double pap = st->pAp;
  const double alpha = (pap > 0.0 && isfinite(pap)) ? st->rr / pap : 0.0;
  const T a = T(alpha);
  double v = 0.0;
  for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * K; i < n; i += (size_t)gridDim.x * blockDim.x * K) {
    cplx<T> rv[K], av[K];
    Chunk<S>::load(r, i / K, rv);
    Chunk<S>::load(Ap, i / K, av);
    T t = T(0);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      rv[c].re = fma(-a, av[c].re, rv[c].re);
      rv[c].im = fma(-a, av[c].im, rv[c].im);
      t += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
    }
    Chunk<S>::store(r, i / K, rv);
    v += (double)t;
  }
  __shared__ double red[32];
  __shared__ double s_tot;
  double s = block_sum_dyn(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (!last_block_done(counter)) return;
  double tot = sum_partials_dyn(partials, gridDim.x, red);
  if (threadIdx.x == 0) {
    s_tot = tot;
    if (!(pap > 0.0)) st->breakdown = 1;
    if (!isfinite(tot)) st->nonfinite = 1;
    st->rr_new = tot;
    st->alpha = alpha;
  }
  __syncthreads();
  // the shifts' recurrences are independent: one thread each (GB300's FP64 divisions are slow in a
  // single thread's dependent chain)
  const double beta = s_tot / st->rr;
  const double s0 = st->sigma[st->base];
  for (int k = threadIdx.x; k < st->nshift; k += blockDim.x) {
    if (!st->active[k]) continue;
    double zn;
    if (k == st->base) {
      zn = 1.0;
    } else {
      const double z = st->zeta[k], zo = st->zeta_old[k];
      const double den = alpha * st->beta_old * (zo - z) + zo * st->alpha_old * (1.0 + (st->sigma[k] - s0) * alpha);
      zn = z * zo * st->alpha_old / den;
    }
    const double ratio = zn / st->zeta[k];
    st->zeta_new[k] = zn;
    st->alpha_k[k] = alpha * ratio;
    st->beta_k[k] = beta * ratio * ratio;
  }
}

// For every active shift: x_k += alpha_k p_k; p_k = zeta_k' r + beta_k p_k (r read once).
// X = double: x_k is the FP64 solution in true units (alpha_k * scale). X = float (FP32 Krylov
// vectors): x_k is an FP32 correction in inner units, folded into the FP64 solutions once the
// Krylov phase ends (k_ms_fold) -- two FP64 operations per entry and shift would otherwise bind this
// streaming kernel to GB300's FP64 pipe. The FP64 verification and refinement that follow the FP32
// Krylov phase correct what the FP32 accumulation loses.
// Last block: commit the recurrences, freeze converged shifts, count the iteration.
template <typename S, typename X>
__global__ void k_ms_update(X* __restrict__ x, S* __restrict__ p, const S* __restrict__ r, size_t n,
                            MsState* st, unsigned* counter) {
  if (st->done) return;
  using T = typename Real<S>::acc;
  using XT = typename Real<X>::acc;
  __shared__ XT s_ax[MAXR];
  __shared__ T s_z[MAXR], s_b[MAXR];
  __shared__ int s_act[MAXR];
  const int ns = st->nshift;
  for (int k = threadIdx.x; k < ns; k += blockDim.x) {
    s_act[k] = st->active[k];
    s_ax[k] = XT(sizeof(X) == 8 ? st->alpha_k[k] * st->scale : st->alpha_k[k]);
    s_z[k] = T(st->zeta_new[k]);
    s_b[k] = T(st->beta_k[k]);
  }
  __syncthreads();
  constexpr int K = Chunk<S>::K;
  for (size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * K; i < n; i += (size_t)gridDim.x * blockDim.x * K) {
    cplx<T> rv[K];
    Chunk<S>::load(r, i / K, rv);
    for (int k = 0; k < ns; ++k) {
      if (!s_act[k]) continue;
      const size_t j = (size_t)k * n + i;
      cplx<T> pv[K];
      cplx<XT> xv[K];
      Chunk<S>::load(p, j / K, pv);
      load_k<X, K>(x, j, xv);
#pragma unroll
      for (int c = 0; c < K; ++c) {
        xv[c].re = fma(s_ax[k], XT(pv[c].re), xv[c].re);
        xv[c].im = fma(s_ax[k], XT(pv[c].im), xv[c].im);
        pv[c].re = fma(s_b[k], pv[c].re, s_z[k] * rv[c].re);
        pv[c].im = fma(s_b[k], pv[c].im, s_z[k] * rv[c].im);
      }
      store_k<X, K>(x, j, xv);
      Chunk<S>::store(p, j / K, pv);
    }
  }
  if (!last_block_done(counter) || threadIdx.x != 0) return;
  st->iter += 1;
  st->cycle_iter += 1;
  st->alpha_old = st->alpha;
  st->beta_old = st->rr_new / st->rr;
  st->rr = st->rr_new;
  const double res2 = st->rr * st->scale * st->scale;
  bool any_other = false;
  for (int k = 0; k < ns; ++k) {
    if (!st->active[k]) continue;
    st->zeta_old[k] = st->zeta[k];
    st->zeta[k] = st->zeta_new[k];
    if (k != st->base && st->zeta[k] * st->zeta[k] * res2 <= st->tol2[k]) {
      st->active[k] = 0;
      st->conv_iter[k] = st->iter;
    }
    if (k != st->base && st->active[k]) any_other = true;
  }
  const int b0 = st->base;
  if (st->active[b0] && !any_other && res2 <= st->tol2[b0]) {
    st->active[b0] = 0;
    st->conv_iter[b0] = st->iter;
  }
  const bool finished = !st->active[b0];
  if (finished || st->cycle_iter >= st->cycle_limit || st->breakdown || st->nonfinite) st->done = 1;
}

// r = b / scale; p_k = r; x_k = 0 (x: the FP64 solutions or the FP32 corrections, see k_ms_update).
template <typename S, typename X>
__global__ void k_ms_init(const double2* __restrict__ b, S* __restrict__ r, S* __restrict__ p, X* __restrict__ x,
                          size_t n, int ns, double inv_scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 bv = b[i];
    const S re = S(bv.x * inv_scale), im = S(bv.y * inv_scale);
    r[2 * i] = re;
    r[2 * i + 1] = im;
    for (int k = 0; k < ns; ++k) {
      const size_t j = (size_t)k * n + i;
      p[2 * j] = re;
      p[2 * j + 1] = im;
      x[2 * j] = X(0);
      x[2 * j + 1] = X(0);
    }
  }
}

// x_k = scale * e_k for every shift: the FP32 corrections of the Krylov phase into the FP64 solutions.
__global__ void k_ms_fold(double2* __restrict__ x, const float2* __restrict__ e, size_t total, const MsState* st) {
  const double scale = st->scale;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = e[i];
    x[i] = make_double2(scale * (double)v.x, scale * (double)v.y);
  }
}

// |b|^2 into out[0] (single rhs).
__global__ void k_norm2(const double2* __restrict__ b, size_t n, double* partials, double* out, unsigned* counter) {
  double v = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 bv = b[i];
    v += bv.x * bv.x + bv.y * bv.y;
  }
  __shared__ double red[32];
  double s = block_sum_dyn(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (last_block_done(counter)) {
    double t = sum_partials_dyn(partials, gridDim.x, red);
    if (threadIdx.x == 0) out[0] = t;
  }
}

template <typename S>
static int ms_iteration(hisq_ctx* ctx, int lp, void* xacc, S* r, S* p, S* Ap, S* t, MsState* st, double* partials,
                        double a_base, int base, int ns) {
  const int sp = sizeof(S) == 8 ? HISQ_F64 : HISQ_F32;
  const size_t n = (size_t)ctx->g.half * 3;
  S* pb = p + (size_t)base * n * 2;
  DslashCall c1;
  c1.out_parity = 1;
  c1.out = t;
  c1.in = pb;
  c1.nrhs = 1;
  c1.rhs_stride = ctx->g.half;
  c1.skip = &st->done;
  int rc = dslash_launch(ctx, lp, sp, c1);
  if (rc != HISQ_OK) return rc;
  DslashCall c2 = c1;
  c2.out_parity = 0;
  c2.out = Ap;
  c2.in = t;
  c2.y = pb;
  c2.a = a_base;
  c2.epi = EPI_AXPY;
  c2.partials = partials + MAXR * partial_stride(ctx);
  c2.dot_out = &st->pAp;
  c2.counter = ctx->d_counters + 6;
  if ((rc = dslash_launch(ctx, lp, sp, c2)) != HISQ_OK) return rc;
  const int grid = blas_grid(ctx, 1, n / Chunk<S>::K, 4).x;  // one thread per 16-byte chunk, one wave
  k_ms_rupdate<S><<<grid, 256, 0, ctx->stream>>>(r, Ap, n, st, partials, partial_stride(ctx), ctx->d_counters + 7);
  using X = typename std::conditional<sizeof(S) == 8, double, float>::type;  // see k_ms_update
  k_ms_update<S, X><<<grid, 256, 0, ctx->stream>>>((X*)xacc, p, r, n, st, ctx->d_counters + 8);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx, 2);
  (void)ns;
  return HISQ_OK;
}

template <typename S>
static int run_multishift(hisq_ctx* ctx, double2* x, const double2* b, int ns, const double* shifts, double mass,
                          const double* tol, int maxiter, const hisq_solver_opts& o, hisq_solver_stats* stats) {
  auto t_start = std::chrono::steady_clock::now();
  const int lp = o.inner_prec;
  const int sp = sizeof(S) == 8 ? HISQ_F64 : HISQ_F32;
  const size_t n = (size_t)ctx->g.half * 3;
  S* r = (S*)workspace(ctx, "ms_r", n * 2 * sizeof(S));
  S* Ap = (S*)workspace(ctx, "ms_Ap", n * 2 * sizeof(S));
  S* t = (S*)workspace(ctx, "ms_t", n * 2 * sizeof(S));
  S* p = (S*)workspace(ctx, "ms_p", (size_t)ns * n * 2 * sizeof(S));
  // the solutions' accumulator during the Krylov phase: x itself (FP64 vectors) or FP32 corrections
  using X = typename std::conditional<sizeof(S) == 8, double, float>::type;
  X* xacc = sizeof(S) == 8 ? (X*)x : (X*)workspace(ctx, "ms_e", (size_t)ns * n * 2 * sizeof(float));
  MsState* st = (MsState*)workspace(ctx, "ms_state", sizeof(MsState));
  double* partials = (double*)workspace(ctx, "ms_partials", 2 * MAXR * partial_stride(ctx) * sizeof(double));
  if (!r || !Ap || !t || !p || !xacc || !st || !partials) return set_error(HISQ_ENOMEM, "multi-shift workspace");
  MsState* h = (MsState*)ctx->pinned;
  int base = 0;
  for (int k = 1; k < ns; ++k)
    if (shifts[k] < shifts[base]) base = k;

  // |b|^2 and the scale of the low-precision Krylov vectors (RMS entry of b -> 1)
  const int grid1 = blas_grid(ctx, 1).x;
  k_norm2<<<grid1, 256, 0, ctx->stream>>>(b, n, partials, (double*)ctx->pinned + 4096, ctx->d_counters + 9);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  const double bb = ((double*)ctx->pinned)[4096];
  if (!isfinite(bb)) return set_error(HISQ_ENONFINITE, "non-finite source");
  if (bb == 0.0) {
    HISQ_CUDA(cudaMemsetAsync(x, 0, (size_t)ns * n * sizeof(double2), ctx->stream));
    return HISQ_OK;
  }
  const double scale = sqrt(bb / (double)n);
  memset(h, 0, sizeof(MsState));
  h->nshift = ns;
  h->base = base;
  h->bb = bb;
  h->rr = bb / (scale * scale);
  h->scale = scale;
  h->alpha_old = 1.0;
  h->beta_old = 0.0;
  h->cycle_limit = o.poll_every;
  for (int k = 0; k < ns; ++k) {
    h->sigma[k] = shifts[k];
    h->zeta[k] = h->zeta_old[k] = 1.0;
    h->active[k] = 1;
    h->conv_iter[k] = -1;
    h->tol2[k] = tol[k] * tol[k] * bb;
  }
  HISQ_CUDA(cudaMemcpyAsync(st, h, sizeof(MsState), cudaMemcpyHostToDevice, ctx->stream));
  k_ms_init<S, X><<<grid1, 256, 0, ctx->stream>>>(b, r, p, xacc, n, ns, 1.0 / scale);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  const double a_base = 4.0 * mass * mass + shifts[base];
  const int cycle = o.poll_every;
  cudaGraphExec_t exec = nullptr;
  long long graph_nodes = 0;
  if (o.use_graph) {
    std::string key = "ms/" + std::to_string(sizeof(S)) + "/" + std::to_string(lp) + "/" + std::to_string(ns) + "/" +
                      std::to_string(base) + "/" + std::to_string(cycle);
    char buf[64];
    for (const void* ptr : {(const void*)x, (const void*)xacc, (const void*)r, (const void*)p, (const void*)Ap,
                            (const void*)t, (const void*)st, (const void*)partials}) {
      snprintf(buf, sizeof buf, "/%p", ptr);
      key += buf;
    }
    snprintf(buf, sizeof buf, "/%a", a_base);
    key += buf;
    auto cached = ctx->graphs.find(key);
    if (cached != ctx->graphs.end()) {
      exec = cached->second.first;
      graph_nodes = cached->second.second;
    } else {
      // tune both Dslash launches of an iteration outside the capture (they are idempotent)
      DslashCall c1;
      c1.out_parity = 1;
      c1.out = t;
      c1.in = p + (size_t)base * n * 2;
      c1.nrhs = 1;
      c1.rhs_stride = ctx->g.half;
      int rc = dslash_launch(ctx, lp, sp, c1);
      if (rc != HISQ_OK) return rc;
      DslashCall c2 = c1;
      c2.out_parity = 0;
      c2.out = Ap;
      c2.in = t;
      c2.y = c1.in;
      c2.a = a_base;
      c2.epi = EPI_AXPY;
      c2.partials = partials + MAXR * partial_stride(ctx);
      c2.dot_out = &st->pAp;
      c2.counter = ctx->d_counters + 6;
      if ((rc = dslash_launch(ctx, lp, sp, c2)) != HISQ_OK) return rc;

      cudaGraph_t graph;
      HISQ_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      ctx->capturing = true;
      int crc = HISQ_OK;
      for (int i = 0; i < cycle && crc == HISQ_OK; ++i)
        crc = ms_iteration<S>(ctx, lp, xacc, r, p, Ap, t, st, partials, a_base, base, ns);
      ctx->capturing = false;
      cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
      if (crc != HISQ_OK) return crc;
      HISQ_CUDA(ce);
      size_t nodes = 0;
      cudaGraphGetNodes(graph, nullptr, &nodes);
      graph_nodes = (long long)nodes;
      ce = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      HISQ_CUDA(ce);
      if (ctx->graphs.size() >= 32) release_graphs(ctx);  // bound the cache
      ctx->graphs[key] = {exec, graph_nodes};
    }
  }
  int status = HISQ_OK;
  int last_iter = 0;
  long long dcalls = 0;
  double dbytes = 0.0;
  for (;;) {
    if (exec) {
      HISQ_CUDA(cudaGraphLaunch(exec, ctx->stream));
      ctx->launches += graph_nodes;
    } else {
      for (int i = 0; i < cycle; ++i) {
        int rc = ms_iteration<S>(ctx, lp, xacc, r, p, Ap, t, st, partials, a_base, base, ns);
        if (rc != HISQ_OK) return rc;
      }
    }
    HISQ_CUDA(cudaMemcpyAsync(h, st, sizeof(MsState), cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    dcalls += 2LL * (h->iter - last_iter);
    dbytes += 2.0 * (h->iter - last_iter) * dslash_bytes(ctx, lp, sp, 1);
    last_iter = h->iter;
    if (h->nonfinite) {
      status = set_error(HISQ_ENONFINITE, "non-finite residual at iteration %d", h->iter);
      break;
    }
    if (h->breakdown) {
      status = set_error(HISQ_EBREAKDOWN, "<p, A p> <= 0 at iteration %d", h->iter);
      break;
    }
    if (!h->active[base]) break;
    if (h->iter >= maxiter) break;  // the verification below reports non-convergence
    h->done = 0;
    h->cycle_iter = 0;
    HISQ_CUDA(cudaMemcpyAsync(&st->done, &h->done, 2 * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  if (sizeof(S) != 8) {  // the FP32 corrections into the FP64 solutions (also on the error paths)
    k_ms_fold<<<grid1, 256, 0, ctx->stream>>>(x, (const float2*)xacc, (size_t)ns * n, st);
    HISQ_CUDA(cudaGetLastError());
    note_launch(ctx);
  }
  if (stats) {
    for (int k = 0; k < ns; ++k) stats->shift_iters[k] = h->conv_iter[k];
    stats->iters = h->iter;
    stats->dslash_calls = dcalls;
    stats->dslash_bytes = dbytes;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  }
  if (status != HISQ_OK) return status;
  const int remaining = maxiter > h->iter ? maxiter - h->iter : 0;
  // Verification in FP64 and, where a shift's true residual misses its tolerance, refinement:
  // one multi-rhs CG over all shifts (per-rhs shift sigma_k, same source), so every link read
  // serves all shifts. Inner precision as requested.
  if (lp == HISQ_F64 || lp == HISQ_DF64) return run_cg<double>(ctx, x, b, 0, ns, mass, shifts, tol, remaining, o, stats);
  return run_cg<float>(ctx, x, b, 0, ns, mass, shifts, tol, remaining, o, stats);
}

// out = a0 b + sum_k a_k x_k (FP64), one pass over b and the nshift solutions.
__global__ void k_rational_combine(double2* __restrict__ out, const double2* __restrict__ b,
                                   const double2* __restrict__ x, size_t n, int ns, double a0,
                                   const double* __restrict__ coeffs) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 bv = b[i];
    double re = a0 * bv.x, im = a0 * bv.y;
    for (int k = 0; k < ns; ++k) {
      const double2 xv = x[(size_t)k * n + i];
      re += coeffs[k] * xv.x;
      im += coeffs[k] * xv.y;
    }
    out[i] = make_double2(re, im);
  }
}

}  // namespace hisq

using namespace hisq;

extern "C" {

int hisq_lanczos_extremes(const double* alpha, const double* beta, int n, double* lmin, double* lmax) {
  if (!alpha || !beta || !lmin || !lmax || n < 1) return set_error(HISQ_EINVAL, "bad argument");
  return lanczos_extremes(alpha, beta, n, lmin, lmax);
}

void hisq_solver_opts_default(hisq_solver_opts* o) {
  if (!o) return;
  o->inner_prec = HISQ_F64;
  o->reliable_period = 50;
  o->use_graph = 1;
  o->poll_every = 25;
  o->reliable_prec = HISQ_F64;
  o->vector_layout = 0;
  o->spinor_prec = HISQ_F32;
}

static int check_solver(hisq_ctx* ctx, const void* x, const void* b, double mass, int maxiter,
                        const hisq_solver_opts* opts, hisq_solver_opts* o) {
  if (!ctx || !x || !b) return set_error(HISQ_EINVAL, "null argument");
  if (!ctx->links_ready) return set_error(HISQ_ENOLINKS, "links not loaded");
  if (!(mass > 0) || maxiter < 0) return set_error(HISQ_EINVAL, "need mass > 0 and maxiter >= 0");
  if ((uintptr_t)x % 16 || (uintptr_t)b % 16) return set_error(HISQ_EINVAL, "vectors must be 16-byte aligned");
  hisq_solver_opts_default(o);
  if (opts) *o = *opts;
  if (o->inner_prec < 0 || o->inner_prec >= NPREC || !ctx->links[o->inner_prec])
    return set_error(HISQ_EINVAL, "inner precision %d not resident", o->inner_prec);
  if ((o->reliable_prec != HISQ_F64 && o->reliable_prec != HISQ_DF64) || !ctx->links[o->reliable_prec])
    return set_error(HISQ_EINVAL, "reliable-update precision %d must be HISQ_F64 or a resident HISQ_DF64",
                     o->reliable_prec);
  if (o->reliable_period < 1 || o->poll_every < 1) return set_error(HISQ_EINVAL, "periods must be >= 1");
  if (o->vector_layout != 0 && o->vector_layout != 1) return set_error(HISQ_EINVAL, "vector_layout must be 0 or 1");
  if (o->inner_prec == HISQ_F64 || o->inner_prec == HISQ_DF64) o->spinor_prec = HISQ_F32;  // unused by plain CG
  const bool sp16 = o->spinor_prec == HISQ_F16 || o->spinor_prec == HISQ_BF16;
  if (o->spinor_prec != HISQ_F32 && !(sp16 && o->spinor_prec == o->inner_prec && o->vector_layout == 0))
    return set_error(HISQ_EINVAL, "spinor_prec %d: HISQ_F32, or 16-bit storage equal to inner_prec with "
                                  "vector_layout 0", o->spinor_prec);
  return HISQ_OK;
}

// Device views of caller vectors: device pointers are used in place; host vectors are
// staged through workspaces and copied back (x only) on exit.
struct Staged {
  double2* x;
  const double2* b;
  bool x_host, b_host;
};

static int stage_solver(hisq_ctx* ctx, double* x, const double* b, size_t xb, size_t bbytes, bool copy_x, Staged* s) {
  s->x_host = !is_device_ptr(x);
  s->b_host = !is_device_ptr(b);
  s->x = s->x_host ? (double2*)workspace(ctx, "user_x", xb) : (double2*)x;
  s->b = s->b_host ? (const double2*)workspace(ctx, "user_b", bbytes) : (const double2*)b;
  if (!s->x || !s->b) return set_error(HISQ_ENOMEM, "staging buffers");
  if (s->x_host && copy_x) HISQ_CUDA(cudaMemcpyAsync(s->x, x, xb, cudaMemcpyHostToDevice, ctx->stream));
  if (s->b_host) HISQ_CUDA(cudaMemcpyAsync((void*)s->b, b, bbytes, cudaMemcpyHostToDevice, ctx->stream));
  return HISQ_OK;
}

static int unstage(hisq_ctx* ctx, double* x, size_t xb, const Staged& s, int rc) {
  if (s.x_host) {
    cudaError_t e = cudaMemcpyAsync(x, s.x, xb, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess && rc == HISQ_OK) return cuda_error(e, "copy-out of x");
  }
  return rc;
}

int hisq_cg(hisq_ctx* ctx, double* x, const double* b, int nrhs, double mass, double rel_tol, int maxiter,
            const hisq_solver_opts* opts, hisq_solver_stats* stats) {
  TraceRange trace("hisq_cg");
  hisq_solver_opts o;
  int rc = check_solver(ctx, x, b, mass, maxiter, opts, &o);
  if (rc != HISQ_OK) return rc;
  if (nrhs < 1 || nrhs > MAXR) return set_error(HISQ_EINVAL, "nrhs %d outside [1, %d]", nrhs, MAXR);
  if (!(rel_tol > 0)) return set_error(HISQ_EINVAL, "rel_tol must be > 0");
  if (stats) memset(stats, 0, sizeof *stats);
  const size_t n = (size_t)ctx->g.half * 3, vb = (size_t)nrhs * n * sizeof(double2);
  Staged s;
  if ((rc = stage_solver(ctx, x, b, vb, vb, true, &s)) != HISQ_OK) return rc;
  std::vector<double> tol(nrhs, rel_tol);
  const long long l0 = ctx->launches;
  if (o.inner_prec == HISQ_F64 || o.inner_prec == HISQ_DF64)
    rc = run_cg<double>(ctx, s.x, s.b, n, nrhs, mass, nullptr, tol.data(), maxiter, o, stats);
  else if (o.spinor_prec == HISQ_F16)
    rc = run_cg<__half>(ctx, s.x, s.b, n, nrhs, mass, nullptr, tol.data(), maxiter, o, stats);
  else if (o.spinor_prec == HISQ_BF16)
    rc = run_cg<__nv_bfloat16>(ctx, s.x, s.b, n, nrhs, mass, nullptr, tol.data(), maxiter, o, stats);
  else
    rc = run_cg<float>(ctx, s.x, s.b, n, nrhs, mass, nullptr, tol.data(), maxiter, o, stats);
  if (stats) stats->kernel_launches = ctx->launches - l0;
  return unstage(ctx, x, vb, s, rc);
}

int hisq_multishift_cg(hisq_ctx* ctx, double* x, const double* b, int nshift, const double* shifts, double mass,
                       const double* rel_tol, int maxiter, const hisq_solver_opts* opts, hisq_solver_stats* stats) {
  TraceRange trace("hisq_multishift_cg");
  hisq_solver_opts o;
  int rc = check_solver(ctx, x, b, mass, maxiter, opts, &o);
  if (rc != HISQ_OK) return rc;
  if (nshift < 1 || nshift > MAXR || !shifts || !rel_tol)
    return set_error(HISQ_EINVAL, "nshift %d outside [1, %d] or null shifts/tolerances", nshift, MAXR);
  if (o.spinor_prec != HISQ_F32) return set_error(HISQ_EINVAL, "multi-shift CG keeps FP32 inner vectors");
  for (int k = 0; k < nshift; ++k)
    if (!(shifts[k] >= 0) || !(rel_tol[k] > 0)) return set_error(HISQ_EINVAL, "shift %d: need sigma >= 0, tol > 0", k);
  if (stats) memset(stats, 0, sizeof *stats);
  const size_t n = (size_t)ctx->g.half * 3;
  Staged s;
  if ((rc = stage_solver(ctx, x, b, (size_t)nshift * n * sizeof(double2), n * sizeof(double2), false, &s)) != HISQ_OK)
    return rc;
  const long long l0 = ctx->launches;
  if (o.inner_prec == HISQ_F64 || o.inner_prec == HISQ_DF64)
    rc = run_multishift<double>(ctx, s.x, s.b, nshift, shifts, mass, rel_tol, maxiter, o, stats);
  else
    rc = run_multishift<float>(ctx, s.x, s.b, nshift, shifts, mass, rel_tol, maxiter, o, stats);
  if (stats) stats->kernel_launches = ctx->launches - l0;
  return unstage(ctx, x, (size_t)nshift * n * sizeof(double2), s, rc);
}


int hisq_rational_apply(hisq_ctx* ctx, double* out, const double* b, double a0, int nshift, const double* shifts,
                        const double* coeffs, double mass, const double* rel_tol, int maxiter,
                        const hisq_solver_opts* opts, hisq_solver_stats* stats) {
  if (!ctx || !out || !b || !coeffs || !shifts || !rel_tol) return set_error(HISQ_EINVAL, "null argument");
  if (nshift < 1 || nshift > MAXR) return set_error(HISQ_EINVAL, "nshift %d outside [1, %d]", nshift, MAXR);
  if ((uintptr_t)out % 16) return set_error(HISQ_EINVAL, "vectors must be 16-byte aligned");
  const size_t n = (size_t)ctx->g.half * 3;
  double2* xs = (double2*)workspace(ctx, "rat_x", (size_t)nshift * n * sizeof(double2));
  double* dc = (double*)workspace(ctx, "rat_coeffs", MAXR * sizeof(double));
  if (!xs || !dc) return set_error(HISQ_ENOMEM, "rational workspace");
  int rc = hisq_multishift_cg(ctx, (double*)xs, b, nshift, shifts, mass, rel_tol, maxiter, opts, stats);
  if (rc != HISQ_OK) return rc;
  const bool bh = !is_device_ptr(b), oh = !is_device_ptr(out);
  const double2* db = (const double2*)b;
  if (bh) {
    double2* t = (double2*)workspace(ctx, "user_b", n * sizeof(double2));
    if (!t) return set_error(HISQ_ENOMEM, "staging");
    HISQ_CUDA(cudaMemcpyAsync(t, b, n * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
    db = t;
  }
  double2* dout = oh ? (double2*)workspace(ctx, "rat_out", n * sizeof(double2)) : (double2*)out;
  if (!dout) return set_error(HISQ_ENOMEM, "staging");
  HISQ_CUDA(cudaMemcpyAsync(dc, coeffs, nshift * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  k_rational_combine<<<ctx->num_sms * 4, 256, 0, ctx->stream>>>(dout, db, xs, n, nshift, a0, dc);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  if (oh) HISQ_CUDA(cudaMemcpyAsync(out, dout, n * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  return HISQ_OK;
}

}  // extern "C"
