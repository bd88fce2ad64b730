// Multi-RHS Dslash on the tensor cores, for FP16 and BF16 storage (links and vectors in the same
// 16-bit type, FP32 accumulation): the form of the paper's multi-RHS Dslash (Sec. 3) in which the n
// right-hand sides make the site's contraction a small dense matrix product.
//
// At an output site x, with the complex 3x3 hop matrices written as real 6x6 blocks and the colour
// vectors as real 6-vectors (re0, im0, re1, im1, re2, im2), the n outputs are
//   out(x)^T [n x 6] = sum over the 16 hops h of in(x+h)^T [n x 6] . M_h^T [6 x 6],
// M_h = +W_mu(x) for a forward hop and -W_mu(x-h)^dag for a backward one. A warp takes one site at a
// time and issues mma.sync.m16n8k16 with M = 16 right-hand sides, N = 8 (6 output reals + 2 zero
// columns), and K = 16 = two hops (the forward and backward hop of one direction and kind, 6 reals + 2
// zero rows each), so 8 products cover the 16 hops of one group of 16 right-hand sides. tcgen05 needs
// M >= 64, which no per-site shape here reaches.
//
// Fragment layout of m16n8k16 (g = lane / 4, q = lane % 4):
//   A: rows g and g+8, columns 2q, 2q+1 (first register pair) and 8+2q, 9+2q: here row = right-hand
//      side, column 2i + {re, im} of colour i = q for the forward hop, 8 + ... for the backward hop;
//      q = 3 is padding.
//   B: rows 2q, 2q+1 (and 8+2q, 9+2q), column g: column g is output real (j = g / 2, re or im),
//      rows are input reals (i = q, re or im); one complex link entry M_ji gives both rows.
//   C: rows g, g+8; columns 2q, 2q+1 = output colour q, (re, im).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dslash_impl.cuh"
#include "tune.h"

namespace hisq {
namespace {

template <typename H>
struct Mma;
template <>
struct Mma<__half> {
  __device__ __forceinline__ static void run(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                             unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  __device__ __forceinline__ static unsigned pack(float re, float im) {
    __half2 h = __floats2half2_rn(re, im);
    return *reinterpret_cast<unsigned*>(&h);
  }
};
template <>
struct Mma<__nv_bfloat16> {
  __device__ __forceinline__ static void run(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                             unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  __device__ __forceinline__ static unsigned pack(float re, float im) {
    __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    return *reinterpret_cast<unsigned*>(&h);
  }
};

// B-fragment word of one hop for output real (j, part) and input colour i, from the entry w of the
// matrix M_ji = +U_ji (forward) or w = U_ij with M_ji = -conj(U_ij) (backward); sign flips and the
// half swap act on the 16-bit fields directly.
__device__ __forceinline__ unsigned bfrag(unsigned w, int part, bool backward) {
  const unsigned sw = __byte_perm(w, 0, 0x1032);  // (im, re)
  if (!backward) return part ? sw : (w ^ 0x80000000u);         // {re, -im} or {im, re}
  return part ? (sw ^ 0x80000000u) : (w ^ 0x80008000u);        // {-re, -im} or {im, -re}
}

// A block of 16 * MT threads takes a tile of MT consecutive output sites at a time and stages, in
// shared memory, the neighbour index and the link of every (hop, site) -- thread (hop, site) -- and
// the vectors of the current group of 16 at every (hop, site) -- thread (vector, site) walks the 16
// hops -- with asynchronous copies, neighbouring threads on neighbouring sites, so the global reads
// are coalesced as in the CUDA-core kernel. Each warp then takes sites of the tile: it reads the
// site's link words and its A fragments (ldmatrix.x4; one 16-byte row per vector: its 3 complex
// colour entries and a zero word) for all 16 hops, then issues the 8 mma of a group of 16 vectors.
// MT output sites per tile (16 or 8), 16 * MT threads per block: fewer sites per tile use less
// shared memory and let more blocks share an SM.
template <int MT>
struct MmaSmem {
  uint4 av[16][MT][16];       // [hop][site][vector slot]: slot = vector ^ (site & 7)
  unsigned lk[16][MT][12];    // [hop][site]: the 9 link entries, rows padded to 48 bytes
  int nb[MT][16];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Asynchronous global -> shared copies (no register holds the data in flight).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <typename H, int MT>
__global__ void __launch_bounds__(16 * MT) dslash_mma_kernel(const DslashKArgs k, int nrhs) {
  constexpr int MMA_THREADS = 16 * MT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MmaSmem<MT>& sm = *reinterpret_cast<MmaSmem<MT>*>(smem_raw);
  if (k.skip && *k.skip) return;
  const Geom& g = k.g;
  const int p = k.out_parity;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, q = lane & 3;
  const int j = gq >> 1, part = gq & 1;
  const bool bval = j < 3 && q < 3;
  const unsigned* in = reinterpret_cast<const unsigned*>(k.in);
  unsigned* out = reinterpret_cast<unsigned*>(k.out);
  const size_t stride = k.rhs_stride;
  const int ntiles = (g.half + MT - 1) / MT;
  // staging roles: site ts of the tile; hop th (neighbour, link) or vector tr (vectors)
  const int ts = tid % MT, th = tid / MT, tr = tid / MT;
  const int hmu = (th >> 1) & 3, hkind = th >> 3, hbwd = th & 1;
  const int hstep = (hkind ? 3 : 1) * (hbwd ? -1 : 1);
  const char* hblk = k.links + (size_t)(((hbwd ? 1 - p : p) * 2 + hkind) * 4 + hmu) * k.blk_bytes;
  const unsigned* hw = reinterpret_cast<const unsigned*>(hblk);
  // ldmatrix.x4 row of this lane: matrix m = lane / 8 (0: forward hop, vectors 0-7; 1: forward, 8-15;
  // 2: backward, 0-7; 3: backward, 8-15), row lane % 8
  const int lm = lane >> 3, lrow = (lane & 7) + (lm & 1) * 8, lhop = lm >> 1;
  // the fourth word of every staged vector row is padding and stays zero
  for (int i = tid; i < 16 * MT * 16; i += MMA_THREADS) (&sm.av[0][0][0])[i] = make_uint4(0u, 0u, 0u, 0u);

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int cb0 = tile * MT;
    const bool svalid = cb0 + ts < g.half;
    {  // neighbour and link of (hop th, site ts)
      int nb = 0;
      if (svalid) {
        int c[4];
        site_coords(g, p, cb0 + ts, c);
        nb = neighbour_cb(g, c, lex_index(g, c), hmu, hstep);
        const int at = hbwd ? nb : cb0 + ts;  // backward links sit at the neighbour
        unsigned* dst = sm.lk[th][ts];
        cp_async16(dst, hw + (size_t)at * 4);
        cp_async16(dst + 4, hw + (size_t)4 * g.half + (size_t)at * 4);
        cp_async4(dst + 8, hw + (size_t)8 * g.half + at);
      } else {
        for (int e = 0; e < 9; ++e) sm.lk[th][ts][e] = 0u;
      }
      sm.nb[ts][th] = nb;
    }
    __syncthreads();
    for (int r0 = 0; r0 < nrhs; r0 += 16) {
      // vectors: thread (tr, ts) copies vector r0 + tr at the 16 neighbours of site ts
      uint4* arow = &sm.av[0][ts][tr ^ (ts & 7)];
      if (svalid && r0 + tr < nrhs) {
        const unsigned* vin = in + (size_t)(r0 + tr) * stride * 3;
#pragma unroll
        for (int hh = 0; hh < 16; ++hh) {
          const unsigned* src = vin + (size_t)sm.nb[ts][hh] * 3;
          unsigned* d = reinterpret_cast<unsigned*>(arow + hh * MT * 16);
          cp_async4(d, src);
          cp_async4(d + 1, src + 1);
          cp_async4(d + 2, src + 2);
        }
      } else {
#pragma unroll
        for (int hh = 0; hh < 16; ++hh) arow[hh * MT * 16] = make_uint4(0u, 0u, 0u, 0u);
      }
      cp_async_wait_all();
      __syncthreads();
#pragma unroll 1
      for (int s = warp; s < MT; s += MMA_THREADS / 32) {
        const int cb = cb0 + s;
        if (cb >= g.half) break;  // warp-uniform
        // all shared-memory reads of the site first (the asm statements keep their order, so the
        // eight ldmatrix are issued back to back and their latencies overlap), then the 8 products
        unsigned a[8][4], b[8][2];
#pragma unroll
        for (int pr = 0; pr < 8; ++pr) {
          b[pr][0] = bval ? bfrag(sm.lk[2 * pr][s][3 * j + q], part, false) : 0u;
          b[pr][1] = bval ? bfrag(sm.lk[2 * pr + 1][s][3 * q + j], part, true) : 0u;
          asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                       : "=r"(a[pr][0]), "=r"(a[pr][1]), "=r"(a[pr][2]), "=r"(a[pr][3])
                       : "r"(smem_u32(&sm.av[2 * pr + lhop][s][lrow ^ (s & 7)])));
        }
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int pr = 0; pr < 8; ++pr) Mma<H>::run(d, a[pr][0], a[pr][1], a[pr][2], a[pr][3], b[pr][0], b[pr][1]);
        if (q < 3) {
          if (r0 + gq < nrhs) out[((size_t)(r0 + gq) * stride + cb) * 3 + q] = Mma<H>::pack(d[0], d[1]);
          if (r0 + gq + 8 < nrhs) out[((size_t)(r0 + gq + 8) * stride + cb) * 3 + q] = Mma<H>::pack(d[2], d[3]);
        }
      }
      __syncthreads();  // the tile's vectors (and, after the last group, its links) are reused next
    }
  }
}

// One tile size as a tuner candidate. The block size is fixed by the tile (16 threads per site), so
// the tuner's block-size argument is ignored and the choice is between the two tile sizes.
template <typename H, int MT>
TuneVariant mma_variant(hisq_ctx* ctx, const DslashKArgs& a, int nrhs) {
  return TuneVariant{(const void*)dslash_mma_kernel<H, MT>, [ctx, &a, nrhs](int) -> cudaError_t {
                       // shared memory above the 48 KB default: a host-side attribute of the function on the
                       // current device, set before every launch (cheap, right on whichever device)
                       cudaError_t e = cudaFuncSetAttribute(dslash_mma_kernel<H, MT>,
                                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                            (int)sizeof(MmaSmem<MT>));
                       if (e != cudaSuccess) return e;
                       int per_sm = 0;
                       cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dslash_mma_kernel<H, MT>, 16 * MT,
                                                                     sizeof(MmaSmem<MT>));
                       const int tiles = (ctx->g.half + MT - 1) / MT;
                       int grid = ctx->num_sms * (per_sm > 0 ? per_sm : 1);
                       if (grid > tiles) grid = tiles;
                       dslash_mma_kernel<H, MT><<<grid, 16 * MT, sizeof(MmaSmem<MT>), ctx->stream>>>(a, nrhs);
                       return cudaGetLastError();
                     }};
}

template <typename H>
int launch_mma_t(hisq_ctx* ctx, int prec, const DslashCall& c) {
  DslashKArgs a;
  a.g = ctx->g;
  a.links = ctx->links[prec];
  a.blk_bytes = link_block_bytes(prec, ctx->g.half);
  a.out_parity = c.out_parity;
  a.out = c.out;
  a.in = c.in;
  a.rhs_stride = c.rhs_stride;
  a.skip = c.skip;
  const int nrhs = c.nrhs;
  char key[48];
  snprintf(key, sizeof key, "dslash_mma/l%d/n%d", prec, nrhs);
  TuneVariant v[2] = {mma_variant<H, 16>(ctx, a, nrhs), mma_variant<H, 8>(ctx, a, nrhs)};
  int vi = 0, block = 0;
  int rc = tuned_variant(ctx, key, v, 2, &vi, &block);
  if (rc != HISQ_OK) return rc;
  HISQ_CUDA(v[vi].run(block));
  note_launch(ctx);
  return HISQ_OK;
}

}  // namespace

// The tensor-core Dslash for 16-bit storage (links and vectors in precision prec), plain epilogue.
int dslash_mma_launch(hisq_ctx* ctx, int prec, const DslashCall& c) {
  if (prec == HISQ_F16) return launch_mma_t<__half>(ctx, prec, c);
  if (prec == HISQ_BF16) return launch_mma_t<__nv_bfloat16>(ctx, prec, c);
  return set_error(HISQ_EINVAL, "tensor-core Dslash: FP16 or BF16 storage only");
}

}  // namespace hisq
