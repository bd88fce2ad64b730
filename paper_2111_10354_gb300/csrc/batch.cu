// Batched mixed-precision CG over many independent lattices of uneven sizes.
//
// Every step of the solve is one launch for all lattices: a persistent grid walks a table of
// tiles (a tile = blockDim consecutive output sites of one lattice), so small and large
// lattices share the GPU without one launch per lattice. Lattices that have met their inner
// tolerance skip their tiles. Reductions are per lattice and deterministic: each tile writes
// its partial, and the CTA that completes a lattice's last tile sums that lattice's partials
// in tile order. One CUDA graph holds a whole reliable cycle -- reliable_period inner
// iterations (FP32 links and spinors, FP32 correction e), the fold x += s e, the FP64 true
// residual and the reliable update -- and the host only replays it and polls once per cycle.
// Tile size (the block size of the batched Dslash) is chosen by the autotuner.
#include <math.h>
#include <string.h>

#include <chrono>
#include <type_traits>
#include <vector>

#include "dslash_impl.cuh"
#include "solver_common.cuh"
#include "trace.h"
#include "tune.h"

namespace hisq {

bool is_device_ptr(const void* p);
double dslash_bytes(const hisq_ctx* ctx, int lp, int sp, int nrhs);

constexpr int MAXB = 256;  // lattices per batch

struct BatchState {
  double rr[MAXB], rr_new[MAXB], pAp[MAXB], bb[MAXB], tol2[MAXB], scale[MAXB], rr_true[MAXB], a[MAXB];
  int done[MAXB];   // frozen for the rest of the cycle (inner tolerance met, or verified)
  int conv[MAXB];   // true FP64 residual verified below tolerance
  int iters[MAXB];  // inner iterations per lattice
  unsigned cnt[6][MAXB];  // per-lattice tile counters, one row per reduction kernel
  unsigned grid_cnt[6];   // per-kernel CTA counters (last CTA does global bookkeeping)
  int nlat, cycle_done, cycle_iter, cycle_limit, breakdown, nonfinite, all_conv, pad;
};

// Device tables describing the batch for one tile size.
struct TileTable {
  int block = 0;
  int ntiles = 0;
  int* tile_lat = nullptr;   // [ntiles]
  int* tile_cb0 = nullptr;   // [ntiles]
  int* lat_tile0 = nullptr;  // [nlat + 1]
};

struct BatchArgs {
  const Geom* geoms;        // [nlat]
  const char* const* links;  // [nlat] link storage of one precision
  const size_t* blk_bytes;   // [nlat]
  const size_t* site_off;    // [nlat] offset of lattice l's vectors, in sites
  const int* tile_lat;
  const int* tile_cb0;
  const int* lat_tile0;
  int ntiles;
  int nlat;
};

// ------------------------------------------------------------------ reduction helpers
// Tile partial -> per-lattice total by the CTA completing the lattice's last tile.
// Returns true (in all threads) in that CTA; thread 0 then holds the total in *total.
__device__ __forceinline__ bool lattice_reduce(double v, int t, int l, const BatchArgs& a, double* partials,
                                               unsigned* cnt, double* red, double* total) {
  __shared__ bool last;
  double s = block_sum_dyn(v, red);
  if (threadIdx.x == 0) partials[t] = s;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned n = (unsigned)(a.lat_tile0[l + 1] - a.lat_tile0[l]);
    last = atomicAdd(&cnt[l], 1u) == n - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double tot = sum_partials_dyn(partials + a.lat_tile0[l], a.lat_tile0[l + 1] - a.lat_tile0[l], red);
  if (threadIdx.x == 0) {
    cnt[l] = 0u;
    *total = tot;
  }
  return true;
}

// True in thread 0 of the last CTA of the grid to reach this point.
__device__ __forceinline__ bool grid_last(unsigned* c) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(c, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    *c = 0u;
  }
  return last && threadIdx.x == 0;
}

// ------------------------------------------------------------------ batched Dslash
// out_l = D in_l (EPI_PLAIN) or out_l = a_l y_l - D in_l with pAp_l = Re<y_l, out_l> (EPI_AXPY),
// for every lattice l whose skip[l] is 0.
template <typename LR, typename SR, int EPI>
__global__ void __launch_bounds__(256) k_bdslash(const BatchArgs a, int p, void* out, const void* in, const void* y,
                                                 const int* skip, BatchState* st, double* partials, int red_row) {
  using A = typename Real<LR>::acc;
  using SA = typename Real<SR>::acc;
  __shared__ double red[32];
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int l = a.tile_lat[t];
    if (skip[l]) continue;  // uniform over the CTA
    const Geom g = a.geoms[l];
    const int cb = a.tile_cb0[t] + threadIdx.x;
    const size_t base = a.site_off[l];
    double dot = 0.0;
    if (cb < g.half) {
      cplx<A> acc[1][3];
      const char* in_l = (const char*)in + base * 6 * sizeof(SR);
      dslash_site<LR, SR, 1>(g, a.links[l], a.blk_bytes[l], p, cb, in_l, 0, acc);
      cplx<SA> o[3];
      if (EPI == EPI_PLAIN) {
#pragma unroll
        for (int i = 0; i < 3; ++i) o[i] = {SA(acc[0][i].re), SA(acc[0][i].im)};
      } else {
        cplx<SA> yv[3];
        VecIO<SR>::load(y, base + cb, yv);
        const A al = A(st->a[l]);
        SA tt = SA(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          o[i].re = SA(fma(al, A(yv[i].re), -acc[0][i].re));
          o[i].im = SA(fma(al, A(yv[i].im), -acc[0][i].im));
          tt += yv[i].re * o[i].re + yv[i].im * o[i].im;
        }
        dot = (double)tt;
      }
      VecIO<SR>::store(out, base + cb, o);
    }
    if (EPI == EPI_AXPY) {
      double tot;
      if (lattice_reduce(dot, t, l, a, partials, st->cnt[red_row], red, &tot) && threadIdx.x == 0) st->pAp[l] = tot;
    }
  }
}

// ------------------------------------------------------------------ batched BLAS-1
// e_l += alpha_l p_l; r_l -= alpha_l Ap_l; rr_new_l = |r_l|^2 (alpha_l = rr_l / pAp_l).
template <typename S, typename X>
__global__ void __launch_bounds__(256) k_bupdate(const BatchArgs a, X* e, S* r, const S* p, const S* Ap,
                                                 BatchState* st, double* partials) {
  if (st->cycle_done) return;
  using T = typename Real<S>::acc;
  using XT = typename Real<X>::acc;
  __shared__ double red[32];
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int l = a.tile_lat[t];
    if (st->done[l]) continue;
    const int half = a.geoms[l].half;
    const int cb = a.tile_cb0[t] + threadIdx.x;
    const size_t site = a.site_off[l] + cb;
    const double pap = st->pAp[l];
    const bool ok = pap > 0.0 && isfinite(pap);
    const double alpha = ok ? st->rr[l] / pap : 0.0;
    double v = 0.0;
    if (cb < half) {
      cplx<T> pv[3], rv[3], av[3];
      cplx<XT> xv[3];
      VecIO<S>::load(p, site, pv);
      VecIO<S>::load(r, site, rv);
      VecIO<S>::load(Ap, site, av);
      VecIO<X>::load(e, site, xv);
      const T al = T(alpha);
      // X = double: e is the FP64 solution itself (true units); X = float: inner units, k_bfold scales
      const XT ax = XT(sizeof(X) == 8 ? alpha * st->scale[l] : alpha);
      T tt = T(0);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xv[c].re = fma(ax, XT(pv[c].re), xv[c].re);
        xv[c].im = fma(ax, XT(pv[c].im), xv[c].im);
        rv[c].re = fma(-al, av[c].re, rv[c].re);
        rv[c].im = fma(-al, av[c].im, rv[c].im);
        tt += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
      }
      VecIO<X>::store(e, site, xv);
      VecIO<S>::store(r, site, rv);
      v = (double)tt;
    }
    double tot;
    if (lattice_reduce(v, t, l, a, partials, st->cnt[1], red, &tot) && threadIdx.x == 0) {
      st->rr_new[l] = tot;
      if (!ok) st->breakdown = 1;
      if (!isfinite(tot)) st->nonfinite = 1;
    }
  }
}

// p_l = r_l + beta_l p_l; per lattice (last tile): commit rr, count the iteration, inner
// convergence; last CTA: end of cycle when every lattice is frozen or the cycle is full.
template <typename S>
__global__ void __launch_bounds__(256) k_bpupdate(const BatchArgs a, const S* r, S* p, BatchState* st) {
  if (st->cycle_done) return;
  using T = typename Real<S>::acc;
  __shared__ bool last;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int l = a.tile_lat[t];
    if (st->done[l]) continue;
    const int half = a.geoms[l].half;
    const int cb = a.tile_cb0[t] + threadIdx.x;
    if (cb < half) {
      const size_t site = a.site_off[l] + cb;
      const T beta = T(st->rr_new[l] / st->rr[l]);
      cplx<T> pv[3], rv[3];
      VecIO<S>::load(p, site, pv);
      VecIO<S>::load(r, site, rv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv[c].re = fma(beta, pv[c].re, rv[c].re);
        pv[c].im = fma(beta, pv[c].im, rv[c].im);
      }
      VecIO<S>::store(p, site, pv);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned n = (unsigned)(a.lat_tile0[l + 1] - a.lat_tile0[l]);
      last = atomicAdd(&st->cnt[2][l], 1u) == n - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      st->cnt[2][l] = 0u;
      st->rr[l] = st->rr_new[l];
      st->iters[l] += 1;
      const double s = st->scale[l];
      if (st->rr[l] * s * s <= st->tol2[l]) st->done[l] = 1;
    }
    __syncthreads();
  }
  if (grid_last(&st->grid_cnt[2])) {
    bool all = true;
    for (int l = 0; l < st->nlat; ++l) all = all && st->done[l];
    st->cycle_iter += 1;
    if (all || st->cycle_iter >= st->cycle_limit || st->breakdown || st->nonfinite) st->cycle_done = 1;
  }
}

// x_l += scale_l e_l; e_l = 0 (all lattices not yet verified).
__global__ void __launch_bounds__(256) k_bfold(const BatchArgs a, double2* x, float* e, BatchState* st) {
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int l = a.tile_lat[t];
    if (st->conv[l]) continue;
    const int cb = a.tile_cb0[t] + threadIdx.x;
    if (cb >= a.geoms[l].half) continue;
    const size_t site = a.site_off[l] + cb;
    const double s = st->scale[l];
    float2* ep = reinterpret_cast<float2*>(e) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 ev = ep[c];
      double2 xv = x[3 * site + c];
      xv.x += s * (double)ev.x;
      xv.y += s * (double)ev.y;
      x[3 * site + c] = xv;
      ep[c] = make_float2(0.f, 0.f);
    }
  }
}

// r_hi = b - Ax (FP64); rr_true and (init) bb per lattice.
__global__ void __launch_bounds__(256) k_bresidual(const BatchArgs a, const double2* b, const double2* Ax, double2* rh,
                                                   BatchState* st, double* partials, int init) {
  __shared__ double red[32];
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int l = a.tile_lat[t];
    if (st->conv[l]) continue;
    const int cb = a.tile_cb0[t] + threadIdx.x;
    double v0 = 0.0, v1 = 0.0;
    if (cb < a.geoms[l].half) {
      const size_t site = a.site_off[l] + cb;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double2 bv = b[3 * site + c], av = Ax[3 * site + c];
        const double2 rv = make_double2(bv.x - av.x, bv.y - av.y);
        rh[3 * site + c] = rv;
        v0 += rv.x * rv.x + rv.y * rv.y;
        v1 += bv.x * bv.x + bv.y * bv.y;
      }
    }
    double tot;
    if (lattice_reduce(v0, t, l, a, partials, st->cnt[3], red, &tot) && threadIdx.x == 0) {
      st->rr_true[l] = tot;
      if (!isfinite(tot)) st->nonfinite = 1;
    }
    if (init) {
      if (lattice_reduce(v1, t, l, a, partials + a.ntiles, st->cnt[4], red, &tot) && threadIdx.x == 0)
        st->bb[l] = tot;
    }
  }
}

// Reliable update per lattice not yet verified: r_lo = r_hi / s, p = r_lo, rr = rr_true / s^2;
// verified lattices are frozen for good. Last CTA: new cycle, or all verified.
template <typename S>
__global__ void __launch_bounds__(256) k_breliable(const BatchArgs a, const double2* rh, S* r, S* p, BatchState* st) {
  __shared__ bool last;
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int l = a.tile_lat[t];
    if (st->conv[l]) continue;
    const int half = a.geoms[l].half;
    const int cb = a.tile_cb0[t] + threadIdx.x;
    const double n = 3.0 * half;
    const bool c = st->rr_true[l] <= st->tol2[l];
    const double s = sqrt(st->rr_true[l] / n);
    if (!c && s > 0.0 && cb < half) {
      const size_t site = a.site_off[l] + cb;
      const double inv = 1.0 / s;
      using T = typename Real<S>::acc;
      cplx<T> v[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 w = rh[3 * site + k];
        v[k] = {T(w.x * inv), T(w.y * inv)};
      }
      VecIO<S>::store(r, site, v);
      VecIO<S>::store(p, site, v);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned nt = (unsigned)(a.lat_tile0[l + 1] - a.lat_tile0[l]);
      last = atomicAdd(&st->cnt[5][l], 1u) == nt - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      st->cnt[5][l] = 0u;
      st->conv[l] = c;
      st->done[l] = c;
      if (!c && s > 0.0) {
        st->scale[l] = s;
        st->rr[l] = st->rr_true[l] / (s * s);
      }
    }
    __syncthreads();
  }
  if (grid_last(&st->grid_cnt[5])) {
    bool all = true;
    for (int l = 0; l < st->nlat; ++l) all = all && st->conv[l];
    st->all_conv = all;
    st->cycle_done = all ? 1 : 0;
    st->cycle_iter = 0;
  }
}

}  // namespace hisq

// ------------------------------------------------------------------ batch object
struct hisq_batch {
  int nlat = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<hisq_ctx*> lat;     // one context per lattice (its links, packing, tuning)
  std::vector<size_t> site_off;   // prefix sums of half
  size_t total_half = 0;
  int num_sms = 0;
  hisq::Geom* d_geoms = nullptr;
  size_t* d_site_off = nullptr;
  const char** d_links[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t* d_blk[4] = {nullptr, nullptr, nullptr, nullptr};
  std::map<int, hisq::TileTable> tiles;  // by tile size
  std::map<std::string, int> tune;
  hisq_ctx* tune_ctx = nullptr;  // borrowed for the tuner's bookkeeping (lattice 0)
  std::map<std::string, DevBuf> ws;
  void* pinned = nullptr;
  long long launches = 0;
};

namespace hisq {

static void* bws(hisq_batch* B, const char* name, size_t bytes) {
  DevBuf& b = B->ws[name];
  if (b.ptr && b.bytes >= bytes) return b.ptr;
  if (b.ptr) {
    cudaStreamSynchronize(B->stream);
    cudaFree(b.ptr);
    b.ptr = nullptr;
  }
  if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    b.bytes = 0;
    return nullptr;
  }
  b.bytes = bytes;
  return b.ptr;
}

static int tile_table(hisq_batch* B, int block, TileTable** out) {
  auto it = B->tiles.find(block);
  if (it != B->tiles.end()) {
    *out = &it->second;
    return HISQ_OK;
  }
  std::vector<int> tl, tc, l0;
  for (int l = 0; l < B->nlat; ++l) {
    l0.push_back((int)tl.size());
    const int half = B->lat[l]->g.half;
    for (int cb = 0; cb < half; cb += block) {
      tl.push_back(l);
      tc.push_back(cb);
    }
  }
  l0.push_back((int)tl.size());
  TileTable T;
  T.block = block;
  T.ntiles = (int)tl.size();
  HISQ_CUDA(cudaMalloc(&T.tile_lat, tl.size() * sizeof(int)));
  HISQ_CUDA(cudaMalloc(&T.tile_cb0, tc.size() * sizeof(int)));
  HISQ_CUDA(cudaMalloc(&T.lat_tile0, l0.size() * sizeof(int)));
  HISQ_CUDA(cudaMemcpy(T.tile_lat, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice));
  HISQ_CUDA(cudaMemcpy(T.tile_cb0, tc.data(), tc.size() * sizeof(int), cudaMemcpyHostToDevice));
  HISQ_CUDA(cudaMemcpy(T.lat_tile0, l0.data(), l0.size() * sizeof(int), cudaMemcpyHostToDevice));
  B->tiles[block] = T;
  *out = &B->tiles[block];
  return HISQ_OK;
}

static BatchArgs batch_args(hisq_batch* B, int prec, const TileTable& T) {
  BatchArgs a;
  a.geoms = B->d_geoms;
  a.links = B->d_links[prec];
  a.blk_bytes = B->d_blk[prec];
  a.site_off = B->d_site_off;
  a.tile_lat = T.tile_lat;
  a.tile_cb0 = T.tile_cb0;
  a.lat_tile0 = T.lat_tile0;
  a.ntiles = T.ntiles;
  a.nlat = B->nlat;
  return a;
}

static int persistent_grid(hisq_batch* B, const void* func, int block) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, block, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return B->num_sms * per_sm;
}

struct BatchBufs {
  double2 *x, *b, *rh, *Ax, *t64;
  void *r, *p, *Ap, *t, *e;
  BatchState* st;
  double* partials;
};

// Launch the batched Dslash in link/spinor type LR/SR with the tuned tile size.
template <typename LR, typename SR, int EPI>
static int bdslash(hisq_batch* B, int p, void* out, const void* in, const void* y, const int* skip, BatchState* st,
                   double* partials, int red_row) {
  auto kern = k_bdslash<LR, SR, EPI>;
  char key[64];
  snprintf(key, sizeof key, "bdslash/l%d/s%d/e%d", Real<LR>::prec, Real<SR>::prec, EPI);
  int block = 0;
  auto it = B->tune.find(key);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HISQ_CUDA(cudaStreamIsCapturing(B->stream, &cap));
  if (it != B->tune.end()) {
    block = it->second;
  } else if (cap != cudaStreamCaptureStatusNone) {
    block = 128;
  } else {
    // autotune the tile size: time each candidate (the launch is idempotent)
    static const int cands[] = {64, 128, 256};
    cudaEvent_t e0, e1;
    HISQ_CUDA(cudaEventCreate(&e0));
    HISQ_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int c : cands) {
      TileTable* T;
      int rc = tile_table(B, c, &T);
      if (rc != HISQ_OK) return rc;
      const BatchArgs a = batch_args(B, Real<LR>::prec, *T);
      const int grid = persistent_grid(B, (const void*)kern, c);
      kern<<<grid, c, 0, B->stream>>>(a, p, out, in, y, skip, st, partials, red_row);
      cudaEventRecord(e0, B->stream);
      for (int r = 0; r < 3; ++r) kern<<<grid, c, 0, B->stream>>>(a, p, out, in, y, skip, st, partials, red_row);
      cudaEventRecord(e1, B->stream);
      B->launches += 4;
      HISQ_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        block = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->tune[key] = block;
  }
  TileTable* T;
  int rc = tile_table(B, block, &T);
  if (rc != HISQ_OK) return rc;
  const BatchArgs a = batch_args(B, Real<LR>::prec, *T);
  kern<<<persistent_grid(B, (const void*)kern, block), block, 0, B->stream>>>(a, p, out, in, y, skip, st, partials,
                                                                            red_row);
  HISQ_CUDA(cudaGetLastError());
  if (cap == cudaStreamCaptureStatusNone) B->launches += 1;
  return HISQ_OK;
}

template <typename S>
static int blas_args(hisq_batch* B, BatchArgs* a, int* grid) {
  TileTable* T;
  int rc = tile_table(B, 256, &T);
  if (rc != HISQ_OK) return rc;
  *a = batch_args(B, HISQ_F64, *T);
  *grid = B->num_sms * 8;
  return HISQ_OK;
}

// r_hi = b - A_64 x for every lattice not yet verified.
static int b_true_residual(hisq_batch* B, const BatchBufs& U, int init) {
  int rc = bdslash<double, double, EPI_PLAIN>(B, 1, U.t64, U.x, nullptr, U.st->conv, U.st, U.partials, 0);
  if (rc != HISQ_OK) return rc;
  // the FP64 A uses a_l from the state and writes pAp, which the inner loop recomputes anyway
  rc = bdslash<double, double, EPI_AXPY>(B, 0, U.Ax, U.t64, U.x, U.st->conv, U.st, U.partials, 0);
  if (rc != HISQ_OK) return rc;
  BatchArgs a;
  int grid;
  if ((rc = blas_args<double>(B, &a, &grid)) != HISQ_OK) return rc;
  k_bresidual<<<grid, 256, 0, B->stream>>>(a, U.b, U.Ax, U.rh, U.st, U.partials, init);
  HISQ_CUDA(cudaGetLastError());
  return HISQ_OK;
}

template <typename S>
static int b_reliable(hisq_batch* B, const BatchBufs& U) {
  BatchArgs a;
  int grid;
  int rc = blas_args<S>(B, &a, &grid);
  if (rc != HISQ_OK) return rc;
  k_breliable<S><<<grid, 256, 0, B->stream>>>(a, U.rh, (S*)U.r, (S*)U.p, U.st);
  HISQ_CUDA(cudaGetLastError());
  return HISQ_OK;
}

template <typename S>
static int b_iteration(hisq_batch* B, const BatchBufs& U, int lp) {
  using X = typename std::conditional<sizeof(S) == 8, double, float>::type;
  int rc;
  if (lp == HISQ_F64) {
    rc = bdslash<double, double, EPI_PLAIN>(B, 1, U.t, U.p, nullptr, U.st->done, U.st, U.partials, 0);
    if (rc == HISQ_OK)
      rc = bdslash<double, double, EPI_AXPY>(B, 0, U.Ap, U.t, U.p, U.st->done, U.st, U.partials, 0);
  } else {
    rc = bdslash<float, float, EPI_PLAIN>(B, 1, U.t, U.p, nullptr, U.st->done, U.st, U.partials, 0);
    if (rc == HISQ_OK) rc = bdslash<float, float, EPI_AXPY>(B, 0, U.Ap, U.t, U.p, U.st->done, U.st, U.partials, 0);
  }
  if (rc != HISQ_OK) return rc;
  BatchArgs a;
  int grid;
  if ((rc = blas_args<S>(B, &a, &grid)) != HISQ_OK) return rc;
  k_bupdate<S, X><<<grid, 256, 0, B->stream>>>(a, (X*)U.e, (S*)U.r, (const S*)U.p, (const S*)U.Ap, U.st,
                                                U.partials + 2 * (size_t)a.ntiles);
  k_bpupdate<S><<<grid, 256, 0, B->stream>>>(a, (const S*)U.r, (S*)U.p, U.st);
  HISQ_CUDA(cudaGetLastError());
  return HISQ_OK;
}

template <typename S>
static int run_batch(hisq_batch* B, double2* x, const double2* b, const double* mass, double tol, int maxiter,
                     const hisq_solver_opts& o, hisq_solver_stats* stats, int* iters_out, double* res_out) {
  auto t0 = std::chrono::steady_clock::now();
  const int lp = o.inner_prec;
  const bool mixed = lp != HISQ_F64;
  const size_t n = B->total_half * 3;
  BatchBufs U;
  U.x = x;
  U.b = const_cast<double2*>(b);
  U.rh = (double2*)bws(B, "rh", n * sizeof(double2));
  U.Ax = (double2*)bws(B, "Ax", n * sizeof(double2));
  U.t64 = (double2*)bws(B, "t64", n * sizeof(double2));
  U.r = bws(B, "r", n * 2 * sizeof(S));
  U.p = bws(B, "p", n * 2 * sizeof(S));
  U.Ap = bws(B, "Ap", n * 2 * sizeof(S));
  U.t = bws(B, "t", n * 2 * sizeof(S));
  U.e = mixed ? bws(B, "e", n * 2 * sizeof(float)) : (void*)x;
  U.st = (BatchState*)bws(B, "state", sizeof(BatchState));
  // partials: 3 rows of one double per tile of the smallest tile size (64)
  size_t max_tiles = 0;
  for (int l = 0; l < B->nlat; ++l) max_tiles += (B->lat[l]->g.half + 63) / 64;
  U.partials = (double*)bws(B, "partials", 4 * max_tiles * sizeof(double));
  if (!U.rh || !U.Ax || !U.t64 || !U.r || !U.p || !U.Ap || !U.t || !U.e || !U.st || !U.partials)
    return set_error(HISQ_ENOMEM, "batch workspace");
  BatchState* h = (BatchState*)B->pinned;
  memset(h, 0, sizeof(BatchState));
  h->nlat = B->nlat;
  h->cycle_limit = mixed ? o.reliable_period : o.poll_every;
  for (int l = 0; l < B->nlat; ++l) {
    h->scale[l] = 1.0;
    h->a[l] = 4.0 * mass[l] * mass[l];
  }
  HISQ_CUDA(cudaMemcpyAsync(U.st, h, sizeof(BatchState), cudaMemcpyHostToDevice, B->stream));
  if (mixed) HISQ_CUDA(cudaMemsetAsync(U.e, 0, n * 2 * sizeof(float), B->stream));
  int rc = b_true_residual(B, U, 1);
  if (rc != HISQ_OK) return rc;
  HISQ_CUDA(cudaMemcpyAsync(h, U.st, sizeof(BatchState), cudaMemcpyDeviceToHost, B->stream));
  HISQ_CUDA(cudaStreamSynchronize(B->stream));
  for (int l = 0; l < B->nlat; ++l) {
    if (!isfinite(h->bb[l]) || !isfinite(h->rr_true[l]))
      return set_error(HISQ_ENONFINITE, "non-finite source or guess in lattice %d", l);
    h->tol2[l] = tol * tol * h->bb[l];
  }
  HISQ_CUDA(cudaMemcpyAsync(U.st->tol2, h->tol2, sizeof(h->tol2), cudaMemcpyHostToDevice, B->stream));
  if ((rc = b_reliable<S>(B, U)) != HISQ_OK) return rc;
  // pre-tune the inner batched Dslash launches outside the capture: they are idempotent (the
  // pAp they write is recomputed by the first iteration before anything reads it)
  if (lp == HISQ_F64) {
    rc = bdslash<double, double, EPI_PLAIN>(B, 1, U.t, U.p, nullptr, U.st->done, U.st, U.partials, 0);
    if (rc == HISQ_OK) rc = bdslash<double, double, EPI_AXPY>(B, 0, U.Ap, U.t, U.p, U.st->done, U.st, U.partials, 0);
  } else {
    rc = bdslash<float, float, EPI_PLAIN>(B, 1, U.t, U.p, nullptr, U.st->done, U.st, U.partials, 0);
    if (rc == HISQ_OK) rc = bdslash<float, float, EPI_AXPY>(B, 0, U.Ap, U.t, U.p, U.st->done, U.st, U.partials, 0);
  }
  if (rc != HISQ_OK) return rc;

  // one graph = one reliable cycle: inner iterations, fold, FP64 residual, reliable update
  const int cycle = h->cycle_limit;
  cudaGraph_t graph;
  cudaGraphExec_t exec = nullptr;
  HISQ_CUDA(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
  int crc = HISQ_OK;
  for (int i = 0; i < cycle && crc == HISQ_OK; ++i) crc = b_iteration<S>(B, U, lp);
  if (crc == HISQ_OK && mixed) {
    BatchArgs a;
    int grid;
    crc = blas_args<S>(B, &a, &grid);
    if (crc == HISQ_OK) k_bfold<<<grid, 256, 0, B->stream>>>(a, U.x, (float*)U.e, U.st);
  }
  if (crc == HISQ_OK) crc = b_true_residual(B, U, 0);
  if (crc == HISQ_OK) crc = b_reliable<S>(B, U);
  cudaError_t ce = cudaStreamEndCapture(B->stream, &graph);
  if (crc != HISQ_OK) return crc;
  HISQ_CUDA(ce);
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  HISQ_CUDA(ce);

  int status = HISQ_OK;
  int cycles = 0;
  HISQ_CUDA(cudaMemcpyAsync(h, U.st, sizeof(BatchState), cudaMemcpyDeviceToHost, B->stream));
  HISQ_CUDA(cudaStreamSynchronize(B->stream));
  while (!h->all_conv) {
    int maxit = 0;
    for (int l = 0; l < B->nlat; ++l) maxit = h->iters[l] > maxit ? h->iters[l] : maxit;
    if (maxit >= maxiter) {
      status = HISQ_ENOCONV;
      break;
    }
    HISQ_CUDA(cudaGraphLaunch(exec, B->stream));
    B->launches += (long long)nodes;
    ++cycles;
    HISQ_CUDA(cudaMemcpyAsync(h, U.st, sizeof(BatchState), cudaMemcpyDeviceToHost, B->stream));
    HISQ_CUDA(cudaStreamSynchronize(B->stream));
    if (h->nonfinite) {
      status = set_error(HISQ_ENONFINITE, "non-finite residual in the batch");
      break;
    }
    if (h->breakdown) {
      status = set_error(HISQ_EBREAKDOWN, "<p, A p> <= 0 in the batch");
      break;
    }
  }
  cudaGraphExecDestroy(exec);
  double worst = 0.0;
  int total_it = 0;
  for (int l = 0; l < B->nlat; ++l) {
    const double rel = h->bb[l] > 0 ? sqrt(h->rr_true[l] / h->bb[l]) : sqrt(h->rr_true[l]);
    worst = rel > worst ? rel : worst;
    total_it = h->iters[l] > total_it ? h->iters[l] : total_it;
    if (iters_out) iters_out[l] = h->iters[l];
    if (res_out) res_out[l] = rel;
  }
  if (stats) {
    stats->iters = total_it;
    stats->reliable_updates = cycles;
    stats->converged = h->all_conv && status == HISQ_OK;
    stats->true_rel_residual = worst;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    double bytes = 0;
    for (int l = 0; l < B->nlat; ++l)
      bytes += 2.0 * h->iters[l] * dslash_bytes(B->lat[l], lp, mixed ? HISQ_F32 : HISQ_F64, 1);
    stats->dslash_bytes = bytes;
  }
  if (status == HISQ_ENOCONV) return set_error(HISQ_ENOCONV, "batch: no convergence in %d iterations", maxiter);
  return status;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

int hisq_batch_create(hisq_batch** out, int nlat, const int* dims, unsigned prec_mask, void* stream) {
  if (!out || !dims || nlat < 1 || nlat > MAXB) return set_error(HISQ_EINVAL, "need 1..%d lattices", MAXB);
  *out = nullptr;
  hisq_batch* B = new (std::nothrow) hisq_batch();
  if (!B) return set_error(HISQ_ENOMEM, "host allocation");
  B->nlat = nlat;
  int rc = HISQ_OK;
  if (stream) {
    B->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreate(&B->stream) != cudaSuccess) {
      delete B;
      return set_error(HISQ_ECUDA, "cudaStreamCreate");
    }
    B->own_stream = true;
  }
  prec_mask |= HISQ_PREC_BIT(HISQ_F64) | HISQ_PREC_BIT(HISQ_F32);
  for (int l = 0; l < nlat && rc == HISQ_OK; ++l) {
    hisq_ctx* c = nullptr;
    rc = hisq_create(&c, dims + 4 * l, prec_mask, B->stream);
    if (rc == HISQ_OK) B->lat.push_back(c);
  }
  if (rc == HISQ_OK) {
    B->num_sms = B->lat[0]->num_sms;
    size_t off = 0;
    std::vector<Geom> geoms;
    for (auto* c : B->lat) {
      B->site_off.push_back(off);
      off += c->g.half;
      geoms.push_back(c->g);
    }
    B->total_half = off;
    cudaError_t e = cudaMalloc(&B->d_geoms, nlat * sizeof(Geom));
    if (e == cudaSuccess) e = cudaMemcpy(B->d_geoms, geoms.data(), nlat * sizeof(Geom), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_site_off, nlat * sizeof(size_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(B->d_site_off, B->site_off.data(), nlat * sizeof(size_t), cudaMemcpyHostToDevice);
    for (int p = 0; p < 4 && e == cudaSuccess; ++p) {
      if (!B->lat[0]->links[p]) continue;
      std::vector<const char*> ptrs;
      std::vector<size_t> blk;
      for (auto* c : B->lat) {
        ptrs.push_back(c->links[p]);
        blk.push_back(link_block_bytes(p, c->g.half));
      }
      e = cudaMalloc(&B->d_links[p], nlat * sizeof(char*));
      if (e == cudaSuccess) e = cudaMemcpy(B->d_links[p], ptrs.data(), nlat * sizeof(char*), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMalloc(&B->d_blk[p], nlat * sizeof(size_t));
      if (e == cudaSuccess) e = cudaMemcpy(B->d_blk[p], blk.data(), nlat * sizeof(size_t), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&B->pinned, sizeof(BatchState) + 4096);
    if (e != cudaSuccess) rc = cuda_error(e, "batch tables");
  }
  if (rc != HISQ_OK) {
    hisq_batch_destroy(B);
    return rc;
  }
  *out = B;
  return HISQ_OK;
}

int hisq_batch_destroy(hisq_batch* B) {
  if (!B) return HISQ_OK;
  if (B->stream) cudaStreamSynchronize(B->stream);
  for (auto* c : B->lat) hisq_destroy(c);
  cudaFree(B->d_geoms);
  cudaFree(B->d_site_off);
  for (int p = 0; p < 4; ++p) {
    cudaFree(B->d_links[p]);
    cudaFree(B->d_blk[p]);
  }
  for (auto& kv : B->tiles) {
    cudaFree(kv.second.tile_lat);
    cudaFree(kv.second.tile_cb0);
    cudaFree(kv.second.lat_tile0);
  }
  for (auto& kv : B->ws) cudaFree(kv.second.ptr);
  if (B->pinned) cudaFreeHost(B->pinned);
  if (B->own_stream) cudaStreamDestroy(B->stream);
  delete B;
  return HISQ_OK;
}

int hisq_batch_load_links(hisq_batch* B, int lattice, const double* fat, const double* lng, unsigned flags) {
  if (!B || lattice < 0 || lattice >= B->nlat) return set_error(HISQ_EINVAL, "bad batch or lattice index");
  return hisq_load_links(B->lat[lattice], fat, lng, flags);
}

long long hisq_batch_vector_offset(const hisq_batch* B, int lattice) {
  if (!B || lattice < 0 || lattice > B->nlat) return -1;
  return lattice == B->nlat ? (long long)B->total_half * 3 : (long long)B->site_off[lattice] * 3;
}

long long hisq_batch_launch_count(const hisq_batch* B) { return B ? B->launches : 0; }

int hisq_batch_cg(hisq_batch* B, double* x, const double* b, const double* mass, double rel_tol, int maxiter,
                  const hisq_solver_opts* opts, hisq_solver_stats* stats, int* iters, double* true_res) {
  TraceRange trace("hisq_batch_cg");
  if (!B || !x || !b || !mass) return set_error(HISQ_EINVAL, "null argument");
  for (int l = 0; l < B->nlat; ++l) {
    if (!B->lat[l]->links_ready) return set_error(HISQ_ENOLINKS, "lattice %d has no links", l);
    if (!(mass[l] > 0)) return set_error(HISQ_EINVAL, "mass of lattice %d must be > 0", l);
  }
  if (!(rel_tol > 0) || maxiter < 0) return set_error(HISQ_EINVAL, "need rel_tol > 0 and maxiter >= 0");
  hisq_solver_opts o;
  hisq_solver_opts_default(&o);
  if (opts) o = *opts;
  if (o.inner_prec != HISQ_F64 && o.inner_prec != HISQ_F32)
    return set_error(HISQ_EINVAL, "batched CG supports FP64 or FP32 inner precision");
  if (o.reliable_period < 1 || o.poll_every < 1) return set_error(HISQ_EINVAL, "periods must be >= 1");
  if ((uintptr_t)x % 16 || (uintptr_t)b % 16) return set_error(HISQ_EINVAL, "vectors must be 16-byte aligned");
  if (stats) memset(stats, 0, sizeof *stats);
  const size_t vb = B->total_half * 3 * sizeof(double2);
  const bool xh = !is_device_ptr(x), bh = !is_device_ptr(b);
  double2* dx = xh ? (double2*)bws(B, "user_x", vb) : (double2*)x;
  const double2* db = bh ? (const double2*)bws(B, "user_b", vb) : (const double2*)b;
  if (!dx || !db) return set_error(HISQ_ENOMEM, "staging");
  if (xh) HISQ_CUDA(cudaMemcpyAsync(dx, x, vb, cudaMemcpyHostToDevice, B->stream));
  if (bh) HISQ_CUDA(cudaMemcpyAsync((void*)db, b, vb, cudaMemcpyHostToDevice, B->stream));
  const long long l0 = B->launches;
  int rc = o.inner_prec == HISQ_F64 ? run_batch<double>(B, dx, db, mass, rel_tol, maxiter, o, stats, iters, true_res)
                                    : run_batch<float>(B, dx, db, mass, rel_tol, maxiter, o, stats, iters, true_res);
  if (stats) stats->kernel_launches = B->launches - l0;
  if (xh) {
    cudaError_t e = cudaMemcpyAsync(x, dx, vb, cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess && rc == HISQ_OK) rc = cuda_error(e, "copy-out");
  }
  return rc;
}

}  // extern "C"
