// C ABI: context life cycle, link loading (fold + pack), Dslash and A dispatch, staging
// of host vectors, errors.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "internal.cuh"
#include "trace.h"
#include "tune.h"

namespace hisq {

int dslash_launch_f64(hisq_ctx* ctx, int sp, const DslashCall& c);
int dslash_launch_f32(hisq_ctx* ctx, int sp, const DslashCall& c);
int dslash_launch_f16(hisq_ctx* ctx, int sp, const DslashCall& c);
int dslash_launch_bf16(hisq_ctx* ctx, int sp, const DslashCall& c);
int dslash_launch_df64(hisq_ctx* ctx, int sp, const DslashCall& c);
int mrhs_launch_f64(hisq_ctx* ctx, int sp, const DslashCall& c);
int mrhs_launch_f32(hisq_ctx* ctx, int sp, const DslashCall& c);
int mrhs_launch_f16(hisq_ctx* ctx, int sp, const DslashCall& c);
int mrhs_launch_bf16(hisq_ctx* ctx, int sp, const DslashCall& c);
int mrhs_launch_df64(hisq_ctx* ctx, int sp, const DslashCall& c);
int dslash_tc_launch(hisq_ctx* ctx, int prec, const DslashCall& c, int* err);

static thread_local char g_last_error[512] = "";

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
  va_end(ap);
  return code;
}

int cuda_error(cudaError_t e, const char* what) {
  set_error(HISQ_ECUDA, "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
  return e == cudaErrorMemoryAllocation ? HISQ_ENOMEM : HISQ_ECUDA;
}

void* workspace(hisq_ctx* ctx, const char* name, size_t bytes) {
  DevBuf& b = ctx->ws[name];
  if (b.bytes >= bytes && b.ptr) return b.ptr;
  if (b.ptr) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    return nullptr;
  }
  b.bytes = bytes;
  return b.ptr;
}

static int dslash_launch_core(hisq_ctx* ctx, int lp, int sp, const DslashCall& c) {
  switch (lp) {
    case HISQ_F64: return dslash_launch_f64(ctx, sp, c);
    case HISQ_F32: return dslash_launch_f32(ctx, sp, c);
    case HISQ_F16: return dslash_launch_f16(ctx, sp, c);
    case HISQ_BF16: return dslash_launch_bf16(ctx, sp, c);
    case HISQ_DF64: return dslash_launch_df64(ctx, sp, c);
  }
  return set_error(HISQ_EINVAL, "bad precision %d", lp);
}

static int mrhs_launch_core(hisq_ctx* ctx, int lp, int sp, const DslashCall& c) {
  switch (lp) {
    case HISQ_F64: return mrhs_launch_f64(ctx, sp, c);
    case HISQ_F32: return mrhs_launch_f32(ctx, sp, c);
    case HISQ_F16: return mrhs_launch_f16(ctx, sp, c);
    case HISQ_BF16: return mrhs_launch_bf16(ctx, sp, c);
    case HISQ_DF64: return mrhs_launch_df64(ctx, sp, c);
  }
  return set_error(HISQ_EINVAL, "bad precision %d", lp);
}

// Interleaved 16-bit storage with 16 or more vectors and the plain epilogue also has a tcgen05
// tensor-core form (dslash_tc.cu). The first call per (precision, rhs count) times both forms (each
// after its own launch-shape tuning; the plain Dslash does not read its output, so running it twice
// is harmless) and keeps the faster: "dslash_path_il/l<prec>/n<nrhs> -> 1 (CUDA cores) or
// 2 (tensor cores)". A bounded tensor-core wait that ran out is reported by that first call (the
// kernel also writes NaN into the affected outputs).
static int dslash_launch_16bit_il(hisq_ctx* ctx, int lp, const DslashCall& c) {
  char key[48];
  snprintf(key, sizeof key, "dslash_path_il/l%d/n%d", lp, c.nrhs);
  int* err = (int*)workspace(ctx, "tc_err", sizeof(int));
  if (!err) return set_error(HISQ_ENOMEM, "tensor-core error flag");
  auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) {
    int v = it->second < 0 ? -it->second : it->second;  // negative: loaded from a report, unchecked
    if (v == 1 || v == 2) {
      it->second = v;
      return v == 2 ? dslash_tc_launch(ctx, lp, c, err) : mrhs_launch_core(ctx, lp, lp, c);
    }
    ctx->tune.erase(it);
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  HISQ_CUDA(cudaStreamIsCapturing(ctx->stream, &cap));
  if (!ctx->autotune || cap != cudaStreamCaptureStatusNone) return mrhs_launch_core(ctx, lp, lp, c);
  HISQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  cudaEvent_t e[2];
  for (auto& ev : e) HISQ_CUDA(cudaEventCreate(&ev));
  float ms[2] = {0.f, 0.f};
  bool ok[2] = {false, false};
  int rc = HISQ_OK;
  for (int path = 0; path < 2; ++path) {
    auto run = [&]() { return path == 1 ? dslash_tc_launch(ctx, lp, c, err) : mrhs_launch_core(ctx, lp, lp, c); };
    rc = run();  // tunes this form's launch shape
    if (rc == HISQ_OK) {
      cudaEventRecord(e[0], ctx->stream);
      rc = run();
      cudaEventRecord(e[1], ctx->stream);
    }
    if (rc == HISQ_OK && cudaEventSynchronize(e[1]) == cudaSuccess) {
      cudaEventElapsedTime(&ms[path], e[0], e[1]);
      ok[path] = true;
    }
    if (!ok[path]) {
      if (path == 0) break;  // the CUDA-core form failed: report it
      cudaGetLastError();    // the tensor-core form could not run here: keep the CUDA-core one
    }
  }
  for (auto& ev : e) cudaEventDestroy(ev);
  if (!ok[0]) return rc != HISQ_OK ? rc : set_error(HISQ_ECUDA, "Dslash timing failed");
  int herr = 0;
  HISQ_CUDA(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) {
    cudaMemsetAsync(err, 0, sizeof(int), ctx->stream);
    ok[1] = false;  // a bounded wait ran out: the tensor-core form is not used
  }
  const bool tensor = ok[1] && ms[1] < ms[0];
  ctx->tune[key] = tensor ? 2 : 1;
  // the output holds the last form's result (both forms agree up to rounding order)
  if (!ok[1]) return mrhs_launch_core(ctx, lp, lp, c);
  return HISQ_OK;
}

int dslash_launch(hisq_ctx* ctx, int lp, int sp, const DslashCall& c) {
  if (!ctx->links[lp]) return set_error(HISQ_EINVAL, "link precision %d is not resident", lp);
  if (c.interleaved) {
    const bool comp = ctx->naik != 0.0 && ctx->long12[lp] != nullptr;
    if ((lp == HISQ_F16 || lp == HISQ_BF16) && sp == lp && c.epi == EPI_PLAIN && c.nrhs >= 16 && c.nrhs <= 64 &&
        c.nrhs % 4 == 0 && !comp)
      return dslash_launch_16bit_il(ctx, lp, c);
    return mrhs_launch_core(ctx, lp, sp, c);
  }
  return dslash_launch_core(ctx, lp, sp, c);
}

double dslash_bytes(const hisq_ctx* ctx, int lp, int sp, int nrhs) {
  // algorithmic: every link once, every vector read once and written once
  return (double)ctx->g.half * (16.0 * 18.0 * real_size(lp) + nrhs * 12.0 * real_size(sp));
}

// ------------------------------------------------------------------ link packing (fold)
// One thread per site of the slab: multiply eta_mu(x) (HISQ_APPLY_PHASES) and the
// antiperiodic-t sign (fat at t = Lt-1, long at t >= Lt-3), then store the link in the
// chunk-plane layout of every resident precision. Non-finite entries raise *bad.
__global__ void pack_links_kernel(Geom g, const double2* __restrict__ fat, const double2* __restrict__ lng, int t0,
                                  int nt, unsigned flags, char* l64, char* l32, char* l16, char* lbf, char* ldf,
                                  int* bad, double naik, char* c32, char* c16, char* cbf) {
  const int slab = g.L[0] * g.L[1] * g.L[2];
  const int n = slab * nt;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    int c[4];
    c[0] = s % g.L[0];
    c[1] = (s / g.L[0]) % g.L[1];
    c[2] = (s / (g.L[0] * g.L[1])) % g.L[2];
    c[3] = t0 + s / slab;
    const int idx = lex_index(g, c);
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const int cb = idx >> 1;
    for (int kind = 0; kind < 2; ++kind) {
      const double2* src = kind == 0 ? fat : lng;
      for (int mu = 0; mu < 4; ++mu) {
        double sign = 1.0;
        if (flags & HISQ_APPLY_PHASES) {
          int sum = 0;
          for (int nu = 0; nu < mu; ++nu) sum += c[nu];
          if (sum & 1) sign = -sign;
        }
        if ((flags & HISQ_ANTIPERIODIC_T) && mu == 3) {
          if (kind == 0 && c[3] == g.L[3] - 1) sign = -sign;
          if (kind == 1 && c[3] >= g.L[3] - 3) sign = -sign;
        }
        cplx<double> U[9];
        bool finite = true;
        for (int k = 0; k < 9; ++k) {
          double2 v = src[((size_t)s * 4 + mu) * 9 + k];
          finite = finite && isfinite(v.x) && isfinite(v.y);
          U[k] = {sign * v.x, sign * v.y};
        }
        if (!finite) atomicOr(bad, 1);
        if (kind == 1 && naik != 0.0 && finite) {
          // compressed copy: the link must be c * V with V in SU(3), c = naik * (its fold sign)
          const double ic = 1.0 / (naik * sign);
          double err = 0.0;
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              double re = 0.0, im = 0.0;
              for (int k = 0; k < 3; ++k) {  // (V V^dag)_ij
                const cplx<double> a = U[3 * i + k], b = U[3 * j + k];
                re += a.re * b.re + a.im * b.im;
                im += a.im * b.re - a.re * b.im;
              }
              re = re * ic * ic - (i == j ? 1.0 : 0.0);
              im = im * ic * ic;
              err = fmax(err, fmax(fabs(re), fabs(im)));
            }
          // det V via row0 . (row1 x row2)
          const cplx<double>* u = U;
          auto mul = [](cplx<double> a, cplx<double> b) { return cplx<double>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; };
          cplx<double> c0 = mul(u[4], u[8]), c1 = mul(u[5], u[7]);
          cplx<double> d0 = {c0.re - c1.re, c0.im - c1.im};
          cplx<double> c2 = mul(u[5], u[6]), c3 = mul(u[3], u[8]);
          cplx<double> d1 = {c2.re - c3.re, c2.im - c3.im};
          cplx<double> c4 = mul(u[3], u[7]), c5 = mul(u[4], u[6]);
          cplx<double> d2 = {c4.re - c5.re, c4.im - c5.im};
          cplx<double> e0 = mul(u[0], d0), e1 = mul(u[1], d1), e2 = mul(u[2], d2);
          const double dre = (e0.re + e1.re + e2.re) * ic * ic * ic - 1.0, dim = (e0.im + e1.im + e2.im) * ic * ic * ic;
          err = fmax(err, fmax(fabs(dre), fabs(dim)));
          if (!(err <= 1e-9)) atomicOr(bad, 2);
          const size_t cblk = (size_t)(par * 4 + mu);
          if (c32) Link12IO<float>::store(c32 + cblk * long12_block_bytes(HISQ_F32, g.half), g.half, cb, U);
          if (c16) Link12IO<__half>::store(c16 + cblk * long12_block_bytes(HISQ_F16, g.half), g.half, cb, U);
          if (cbf) Link12IO<__nv_bfloat16>::store(cbf + cblk * long12_block_bytes(HISQ_BF16, g.half), g.half, cb, U);
        }
        const size_t blk = (size_t)((par * 2 + kind) * 4 + mu);
        if (l64) LinkIO<double>::store(l64 + blk * link_block_bytes(HISQ_F64, g.half), g.half, cb, U);
        if (l32) LinkIO<float>::store(l32 + blk * link_block_bytes(HISQ_F32, g.half), g.half, cb, U);
        if (l16) LinkIO<__half>::store(l16 + blk * link_block_bytes(HISQ_F16, g.half), g.half, cb, U);
        if (lbf) LinkIO<__nv_bfloat16>::store(lbf + blk * link_block_bytes(HISQ_BF16, g.half), g.half, cb, U);
        if (ldf) LinkIO<df64>::store(ldf + blk * link_block_bytes(HISQ_DF64, g.half), g.half, cb, U);
      }
    }
  }
}

int pack_links_slab(hisq_ctx* ctx, const double* d_fat, const double* d_long, int t0, int nt, unsigned flags) {
  const int n = ctx->g.L[0] * ctx->g.L[1] * ctx->g.L[2] * nt;
  const int block = 128;
  int grid = (n + block - 1) / block;
  if (grid > ctx->num_sms * 32) grid = ctx->num_sms * 32;
  pack_links_kernel<<<grid, block, 0, ctx->stream>>>(ctx->g, (const double2*)d_fat, (const double2*)d_long, t0, nt,
                                                     flags, ctx->links[0], ctx->links[1], ctx->links[2],
                                                     ctx->links[3], ctx->links[4], ctx->d_flag, ctx->naik, ctx->long12[1],
                                                     ctx->long12[2], ctx->long12[3]);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  return HISQ_OK;
}

// ------------------------------------------------------------------ vector staging
void release_graphs(hisq_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.first);
  ctx->graphs.clear();
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace hisq

using namespace hisq;

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* hisq_strerror(int code) {
  switch (code) {
    case HISQ_OK: return "success";
    case HISQ_EINVAL: return "invalid argument";
    case HISQ_ENOLINKS: return "links not loaded";
    case HISQ_ENOMEM: return "out of memory";
    case HISQ_ECUDA: return "CUDA error";
    case HISQ_ENONFINITE: return "non-finite value";
    case HISQ_ENOCONV: return "solver did not converge";
    case HISQ_EBREAKDOWN: return "solver breakdown";
    case HISQ_ETIMEOUT: return "device wait timed out";
  }
  return "unknown error";
}

const char* hisq_last_error(void) { return g_last_error; }

int hisq_create(hisq_ctx** out, const int dims[4], unsigned prec_mask, void* stream) {
  if (!out || !dims) return set_error(HISQ_EINVAL, "null argument");
  *out = nullptr;
  long long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 4 || (dims[m] & 1)) return set_error(HISQ_EINVAL, "extent %d of dimension %d must be even and >= 4", dims[m], m);
    V *= dims[m];
  }
  if (V > (1LL << 30)) return set_error(HISQ_EINVAL, "volume %lld too large (max 2^30 sites)", V);
  if (prec_mask & ~HISQ_PREC_ALL) return set_error(HISQ_EINVAL, "bad precision mask 0x%x", prec_mask);
  hisq_ctx* c = new (std::nothrow) hisq_ctx();
  if (!c) return set_error(HISQ_ENOMEM, "host allocation");
  for (int m = 0; m < 4; ++m) c->g.L[m] = dims[m];
  c->g.stride[0] = 1;
  c->g.stride[1] = dims[0];
  c->g.stride[2] = dims[0] * dims[1];
  c->g.stride[3] = dims[0] * dims[1] * dims[2];
  c->g.half_x = dims[0] / 2;
  c->g.V = (int)V;
  c->g.half = (int)(V / 2);
  c->prec_mask = prec_mask | HISQ_PREC_BIT(HISQ_F64);
  c->t_loaded.assign(dims[3], 0);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  c->device = dev;
  if (e != cudaSuccess) {
    delete c;
    return cuda_error(e, "device query");
  }
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    // A blocking stream: ordered with the legacy default stream, and capturable.
    e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) {
      delete c;
      return cuda_error(e, "cudaStreamCreate");
    }
    c->own_stream = true;
  }
  int rc = HISQ_OK;
  for (int p = 0; p < NPREC && rc == HISQ_OK; ++p) {
    if (!(c->prec_mask & HISQ_PREC_BIT(p))) continue;
    size_t bytes = 16 * link_block_bytes(p, c->g.half);
    e = cudaMalloc((void**)&c->links[p], bytes);
    if (e != cudaSuccess) rc = cuda_error(e, "link storage");
  }
  if (rc == HISQ_OK) {
    e = cudaMalloc((void**)&c->d_counters, 64 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, 64 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_flag, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->pinned, 1 << 16);
    if (e != cudaSuccess) rc = cuda_error(e, "context buffers");
  }
  if (rc != HISQ_OK) {
    hisq_destroy(c);
    return rc;
  }
  *out = c;
  return HISQ_OK;
}

int hisq_destroy(hisq_ctx* c) {
  if (!c) return HISQ_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (int p = 0; p < NPREC; ++p) {
    cudaFree(c->links[p]);
    cudaFree(c->long12[p]);
  }
  release_graphs(c);
  for (auto& kv : c->ws) cudaFree(kv.second.ptr);
  cudaFree(c->d_counters);
  cudaFree(c->d_flag);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return HISQ_OK;
}

int hisq_load_links_slab(hisq_ctx* c, int t_begin, int t_count, const double* fat, const double* lng,
                         unsigned flags) {
  TraceRange trace("hisq_load_links_slab");
  if (!c || !fat || !lng) return set_error(HISQ_EINVAL, "null argument");
  if (t_begin < 0 || t_count < 1 || t_begin + t_count > c->g.L[3])
    return set_error(HISQ_EINVAL, "t-slab [%d, %d) outside [0, %d)", t_begin, t_begin + t_count, c->g.L[3]);
  if (flags & ~(HISQ_APPLY_PHASES | HISQ_ANTIPERIODIC_T)) return set_error(HISQ_EINVAL, "bad flags 0x%x", flags);
  bool any = false;
  for (unsigned char v : c->t_loaded) any = any || v;
  if (any && flags != c->load_flags) return set_error(HISQ_EINVAL, "flags differ from the slabs already loaded");
  c->load_flags = flags;
  const size_t slice = (size_t)c->g.L[0] * c->g.L[1] * c->g.L[2] * 4 * 9 * 2;  // doubles per t-slice
  // chunks of t-slices bounded to ~512 MB of staging per kind
  int chunk = (int)((512u << 20) / (slice * sizeof(double)));
  if (chunk < 1) chunk = 1;
  if (chunk > t_count) chunk = t_count;
  double* d_fat = (double*)workspace(c, "stage_fat", chunk * slice * sizeof(double));
  double* d_long = (double*)workspace(c, "stage_long", chunk * slice * sizeof(double));
  if (!d_fat || !d_long) return set_error(HISQ_ENOMEM, "link staging buffers");
  HISQ_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  c->links_ready = false;
  for (int t = 0; t < t_count; t += chunk) {
    int nt = t + chunk <= t_count ? chunk : t_count - t;
    size_t off = (size_t)t * slice;
    HISQ_CUDA(cudaMemcpyAsync(d_fat, fat + off, nt * slice * sizeof(double), cudaMemcpyDefault, c->stream));
    HISQ_CUDA(cudaMemcpyAsync(d_long, lng + off, nt * slice * sizeof(double), cudaMemcpyDefault, c->stream));
    int rc = pack_links_slab(c, d_fat, d_long, t_begin + t, nt, flags);
    if (rc != HISQ_OK) return rc;
  }
  int bad = 0;
  HISQ_CUDA(cudaMemcpyAsync(&bad, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HISQ_CUDA(cudaStreamSynchronize(c->stream));
  if (bad) {
    for (auto& v : c->t_loaded) v = 0;
    if (bad & 1)
      return set_error(HISQ_ENONFINITE, "non-finite link entries in t-slab [%d, %d)", t_begin, t_begin + t_count);
    return set_error(HISQ_EINVAL, "long links in t-slab [%d, %d) are not naik * SU(3): they cannot be compressed",
                     t_begin, t_begin + t_count);
  }
  for (int t = t_begin; t < t_begin + t_count; ++t) c->t_loaded[t] = 1;
  bool all = true;
  for (unsigned char v : c->t_loaded) all = all && v;
  c->links_ready = all;
  return HISQ_OK;
}

int hisq_load_links(hisq_ctx* c, const double* fat, const double* lng, unsigned flags) {
  if (!c) return set_error(HISQ_EINVAL, "null context");
  for (auto& v : c->t_loaded) v = 0;
  return hisq_load_links_slab(c, 0, c->g.L[3], fat, lng, flags);
}

static int check_vec_args(hisq_ctx* c, int prec, int nrhs) {
  if (!c) return set_error(HISQ_EINVAL, "null context");
  if (prec < 0 || prec >= NPREC) return set_error(HISQ_EINVAL, "bad precision %d", prec);
  if (!c->links[prec]) return set_error(HISQ_EINVAL, "precision %d not resident", prec);
  if (nrhs < 1 || nrhs > 64) return set_error(HISQ_EINVAL, "nrhs %d outside [1, 64]", nrhs);
  if (!c->links_ready) return set_error(HISQ_ENOLINKS, "links not loaded");
  return HISQ_OK;
}

static size_t vec_bytes(const hisq_ctx* c, int prec, int nrhs) {
  return (size_t)nrhs * c->g.half * 6 * real_size(prec);
}

static bool aligned(const void* p, int prec) {
  size_t a = (prec == HISQ_F64 || prec == HISQ_DF64) ? 16 : prec == HISQ_F32 ? 8 : 4;
  return ((uintptr_t)p % a) == 0;
}

// Resolve a possibly-host vector to a device pointer (copying host input in).
static int stage_in(hisq_ctx* c, const void* p, size_t bytes, const char* name, const void** dev) {
  if (is_device_ptr(p)) {
    *dev = p;
    return HISQ_OK;
  }
  void* d = workspace(c, name, bytes);
  if (!d) return set_error(HISQ_ENOMEM, "staging buffer %s", name);
  HISQ_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, c->stream));
  *dev = d;
  return HISQ_OK;
}

static int dslash_entry(hisq_ctx* c, int out_parity, void* out, const void* in, int prec, int nrhs,
                        bool interleaved) {
  int rc = check_vec_args(c, prec, nrhs);
  if (rc != HISQ_OK) return rc;
  if (out_parity != 0 && out_parity != 1) return set_error(HISQ_EINVAL, "parity %d", out_parity);
  if (!out || !in || out == in) return set_error(HISQ_EINVAL, "null or aliased vectors");
  if (!aligned(out, prec) || !aligned(in, prec)) return set_error(HISQ_EINVAL, "misaligned vector");
  const size_t bytes = vec_bytes(c, prec, nrhs);
  const void* d_in;
  if ((rc = stage_in(c, in, bytes, "stage_in", &d_in)) != HISQ_OK) return rc;
  bool host_out = !is_device_ptr(out);
  void* d_out = host_out ? workspace(c, "stage_out", bytes) : out;
  if (!d_out) return set_error(HISQ_ENOMEM, "staging buffer");
  DslashCall call;
  call.out_parity = out_parity;
  call.out = d_out;
  call.in = d_in;
  call.nrhs = nrhs;
  call.rhs_stride = c->g.half;
  call.interleaved = interleaved;
  rc = dslash_launch(c, prec, prec, call);
  if (rc != HISQ_OK) return rc;
  if (host_out) {
    HISQ_CUDA(cudaMemcpyAsync(out, d_out, bytes, cudaMemcpyDeviceToHost, c->stream));
    HISQ_CUDA(cudaStreamSynchronize(c->stream));
  }
  return HISQ_OK;
}

static int apply_A_entry(hisq_ctx* c, void* out, const void* in, double mass, double sigma, int prec, int nrhs,
                         bool interleaved) {
  int rc = check_vec_args(c, prec, nrhs);
  if (rc != HISQ_OK) return rc;
  if (!out || !in || out == in) return set_error(HISQ_EINVAL, "null or aliased vectors");
  if (!aligned(out, prec) || !aligned(in, prec)) return set_error(HISQ_EINVAL, "misaligned vector");
  if (!(mass >= 0) || !(sigma >= 0)) return set_error(HISQ_EINVAL, "mass and sigma must be >= 0");
  const size_t bytes = vec_bytes(c, prec, nrhs);
  const void* d_in;
  if ((rc = stage_in(c, in, bytes, "stage_in", &d_in)) != HISQ_OK) return rc;
  bool host_out = !is_device_ptr(out);
  void* d_out = host_out ? workspace(c, "stage_out", bytes) : out;
  void* tmp = workspace(c, "apply_tmp", bytes);
  if (!d_out || !tmp) return set_error(HISQ_ENOMEM, "workspace");
  DslashCall c1;
  c1.out_parity = 1;
  c1.out = tmp;
  c1.in = d_in;
  c1.nrhs = nrhs;
  c1.rhs_stride = c->g.half;
  c1.interleaved = interleaved;
  if ((rc = dslash_launch(c, prec, prec, c1)) != HISQ_OK) return rc;
  DslashCall c2 = c1;
  c2.out_parity = 0;
  c2.out = d_out;
  c2.in = tmp;
  c2.y = d_in;
  c2.a = 4.0 * mass * mass + sigma;
  c2.epi = EPI_AXPY;
  if ((rc = dslash_launch(c, prec, prec, c2)) != HISQ_OK) return rc;
  if (host_out) {
    HISQ_CUDA(cudaMemcpyAsync(out, d_out, bytes, cudaMemcpyDeviceToHost, c->stream));
    HISQ_CUDA(cudaStreamSynchronize(c->stream));
  }
  return HISQ_OK;
}

int hisq_dslash(hisq_ctx* c, int out_parity, void* out, const void* in, int prec, int nrhs) {
  return dslash_entry(c, out_parity, out, in, prec, nrhs, false);
}

int hisq_dslash_interleaved(hisq_ctx* c, int out_parity, void* out, const void* in, int prec, int nrhs) {
  return dslash_entry(c, out_parity, out, in, prec, nrhs, true);
}

int hisq_apply_A(hisq_ctx* c, void* out, const void* in, double mass, double sigma, int prec, int nrhs) {
  return apply_A_entry(c, out, in, mass, sigma, prec, nrhs, false);
}

int hisq_apply_A_interleaved(hisq_ctx* c, void* out, const void* in, double mass, double sigma, int prec,
                             int nrhs) {
  return apply_A_entry(c, out, in, mass, sigma, prec, nrhs, true);
}

long long hisq_launch_count(const hisq_ctx* c) { return c ? c->launches : 0; }

int hisq_set_long_compression(hisq_ctx* c, double naik) {
  if (!c) return set_error(HISQ_EINVAL, "null context");
  if (!(naik == naik) || fabs(naik) > 1e6) return set_error(HISQ_EINVAL, "bad Naik coefficient");
  if (naik == c->naik) return HISQ_OK;
  cudaStreamSynchronize(c->stream);
  release_graphs(c);  // captured Dslash launches carry the compression state
  for (int p = 1; p < 4; ++p) {
    cudaFree(c->long12[p]);
    c->long12[p] = nullptr;
    if (naik != 0.0 && c->links[p]) {
      cudaError_t e = cudaMalloc((void**)&c->long12[p], 8 * long12_block_bytes(p, c->g.half));
      if (e != cudaSuccess) {
        c->naik = 0.0;
        return cuda_error(e, "compressed long-link storage");
      }
    }
  }
  c->naik = naik;
  // the compressed copy is written when links are loaded: links must be (re)loaded now
  for (auto& v : c->t_loaded) v = 0;
  c->links_ready = false;
  return HISQ_OK;
}

double hisq_dslash_bytes(const hisq_ctx* c, int prec, int nrhs) {
  if (!c || prec < 0 || prec >= NPREC) return 0.0;
  return dslash_bytes(c, prec, prec, nrhs);
}

int hisq_set_autotune(hisq_ctx* c, int enable) {
  if (!c) return set_error(HISQ_EINVAL, "null context");
  c->autotune = enable ? 1 : 0;
  return HISQ_OK;
}

int hisq_set_pdl(hisq_ctx* c, int enable) {
  if (!c) return set_error(HISQ_EINVAL, "null context");
  c->pdl = enable ? 1 : 0;
  return HISQ_OK;
}

int hisq_tune_load(hisq_ctx* c, const char* report, int* loaded) {
  if (!c || !report) return set_error(HISQ_EINVAL, "null argument");
  int n = 0;
  const char* line = report;
  while (*line) {
    const char* end = strchr(line, '\n');
    const size_t len = end ? (size_t)(end - line) : strlen(line);
    if (len > 0) {
      char key[128];
      int L[4], value;
      const std::string text(line, len);
      if (sscanf(text.c_str(), "%127s %dx%dx%dx%d -> %d", key, &L[0], &L[1], &L[2], &L[3], &value) != 6 ||
          value < 1)
        return set_error(HISQ_EINVAL, "malformed tune line: %.80s", text.c_str());
      if (L[0] == c->g.L[0] && L[1] == c->g.L[1] && L[2] == c->g.L[2] && L[3] == c->g.L[3]) {
        c->tune[key] = -value;  // checked against the kernel's launch forms at first use
        ++n;
      }
    }
    if (!end) break;
    line = end + 1;
  }
  if (loaded) *loaded = n;
  return HISQ_OK;
}

int hisq_release_workspaces(hisq_ctx* c) {
  if (!c) return set_error(HISQ_EINVAL, "null context");
  HISQ_CUDA(cudaStreamSynchronize(c->stream));
  release_graphs(c);  // they were captured on workspace pointers
  for (auto& kv : c->ws) cudaFree(kv.second.ptr);
  c->ws.clear();
  HISQ_CUDA(cudaGetLastError());
  return HISQ_OK;
}

int hisq_tune_report(const hisq_ctx* c, char* buf, size_t len) {
  if (!c || !buf || len == 0) return set_error(HISQ_EINVAL, "null argument");
  size_t used = 0;
  buf[0] = 0;
  for (auto& kv : c->tune) {
    int n = snprintf(buf + used, len - used, "%s %dx%dx%dx%d -> %d\n", kv.first.c_str(), c->g.L[0], c->g.L[1],
                     c->g.L[2], c->g.L[3], kv.second < 0 ? -kv.second : kv.second);
    if (n < 0 || (size_t)n >= len - used) break;
    used += n;
  }
  return HISQ_OK;
}

}  // extern "C"
