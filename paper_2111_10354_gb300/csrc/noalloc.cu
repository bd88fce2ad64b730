// hisq_apply_A_noalloc: the shifted operator of hisq_apply_A for callers that cannot allocate
// device memory at the time of the call. hisq_apply_A keeps the odd-site intermediate
// D_oe in in a context workspace that it allocates with cudaMalloc on first use (and grows
// when a larger nrhs arrives). Some callers cannot allow that: code whose device memory is
// owned by an allocator that forbids foreign allocations, and latency-critical loops that
// cannot take cudaMalloc's implicit device synchronisation.
// This entry point keeps the intermediate in a fixed file-scope device array instead and
// allocates nothing; the caller passes device input and output as usual.
#include <mutex>

#include "internal.cuh"

namespace hisq {

int dslash_launch(hisq_ctx* ctx, int lp, int sp, const DslashCall& c);
bool is_device_ptr(const void* p);

// Scratch for the odd-site intermediate. Every GPU that loads the library holds these
// HISQ_NOALLOC_SCRATCH_BYTES until the process exits. All calls share it: calls whose
// work overlaps on the GPU (several streams, or several host threads) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HISQ_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device. In host code the array's name is only a
// host-side stand-in, so the address is looked up once per device, with that device current.
static void* g_scratch_addr[64];
static std::mutex g_scratch_mutex;

// The array is looked up on the context's own device: the launches run on the context's stream,
// whose device holds the links, so a copy of the array on any other device would be out of reach.
static int scratch_address(const hisq_ctx* c, void** out) {
  int dev = -1;
  HISQ_CUDA(cudaGetDevice(&dev));
  if (dev != c->device)
    return set_error(HISQ_EINVAL, "the current device %d is not the context's device %d", dev, c->device);
  if (dev < 0 || dev >= 64) return set_error(HISQ_EINVAL, "device ordinal %d outside [0, 64)", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HISQ_OK;
}

}  // namespace hisq

using namespace hisq;

extern "C" int hisq_apply_A_noalloc(hisq_ctx* c, void* out, const void* in, double mass, double sigma, int prec,
                                    int nrhs) {
  if (!c) return set_error(HISQ_EINVAL, "null context");
  if (prec < 0 || prec >= NPREC || !c->links[prec]) return set_error(HISQ_EINVAL, "precision %d not resident", prec);
  if (nrhs < 1 || nrhs > 64) return set_error(HISQ_EINVAL, "nrhs %d outside [1, 64]", nrhs);
  if (!c->links_ready) return set_error(HISQ_ENOLINKS, "links not loaded");
  if (!out || !in || out == in) return set_error(HISQ_EINVAL, "null or aliased vectors");
  if (!is_device_ptr(out) || !is_device_ptr(in))
    return set_error(HISQ_EINVAL, "hisq_apply_A_noalloc takes device vectors only (host staging would allocate)");
  const size_t align = (prec == HISQ_F64 || prec == HISQ_DF64) ? 16 : prec == HISQ_F32 ? 8 : 4;
  if ((uintptr_t)out % align || (uintptr_t)in % align) return set_error(HISQ_EINVAL, "misaligned vector");
  if (!(mass >= 0) || !(sigma >= 0)) return set_error(HISQ_EINVAL, "mass and sigma must be >= 0");
  const size_t need = (size_t)nrhs * c->g.half * 6 * real_size(prec);
  if (need > (size_t)HISQ_NOALLOC_SCRATCH_BYTES)
    return set_error(HISQ_EINVAL, "needs %zu bytes of scratch for the odd-site intermediate; the fixed maximum is %zu",
                     need, (size_t)HISQ_NOALLOC_SCRATCH_BYTES);
  void* tmp = nullptr;
  int rc = scratch_address(c, &tmp);
  if (rc != HISQ_OK) return rc;
  // tmp is written in full by the first launch before the second reads it: nothing to clear.
  DslashCall c1;
  c1.out_parity = 1;
  c1.out = tmp;
  c1.in = in;
  c1.nrhs = nrhs;
  c1.rhs_stride = c->g.half;
  if ((rc = dslash_launch(c, prec, prec, c1)) != HISQ_OK) return rc;
  DslashCall c2 = c1;
  c2.out_parity = 0;
  c2.out = out;
  c2.in = tmp;
  c2.y = in;
  c2.a = 4.0 * mass * mass + sigma;
  c2.epi = EPI_AXPY;
  return dslash_launch(c, prec, prec, c2);
}
