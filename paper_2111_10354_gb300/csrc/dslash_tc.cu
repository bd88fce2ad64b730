// Multi-RHS Dslash on the fifth-generation tensor cores (tcgen05) for 16-bit storage, on the
// rhs-interleaved vector layout [cb][color][rhs] (the multi-RHS form of Sec. 3).
//
// At one output site the operator is a small dense contraction over the 16 hops,
//   out[r][i] = sum_h sum_j W_h[i][j] v_h[r][j],   W_h = F or L (forward), -F^dag or -L^dag (backward),
// which in real arithmetic is D[r][n] = sum_k A[r][k] B[n][k] with M = the vectors r (up to 64),
// N = 8 (the 6 output reals, two zero rows) and K = 16 hops x 8 (each hop's 6 input reals and two
// zeros). One CTA takes SITES output sites per round:
//   - A (one 64 x 128 K-major tile per site): the threads gather each neighbour's colour words (rows
//     of nrhs 4-byte (re, im) pairs, coalesced) with asynchronous copies into one 16-byte row per
//     vector and hop;
//   - B (one 8 x 128 tile per site): each hop's link in real form, built with sign flips and half
//     swaps of its 16-bit words (exact: the links are stored in the same 16-bit format);
//   - one thread issues 8 tcgen05.mma (M = 64, N = 8, K = 16) per site into 8 TMEM columns of the
//     site, commits to an mbarrier, and every thread waits for it (bounded);
//   - the accumulators are read back with tcgen05.ld (row r of an M = 64 tile sits in TMEM lane
//     32 (r / 16) + r % 16) and stored as 16-bit pairs.
// Every wait is bounded; on expiry the kernel sets the error flag, writes NaN into the round's
// output, lets the outstanding MMAs drain, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.cuh"
#include "tc.cuh"

namespace hisq {

constexpr int TCD_SITES = 4;                    // output sites per round
constexpr int TCD_A_BYTES = 64 * 128 * 2;       // one site's A tile: 64 rows x 128 K, 16-bit
constexpr int TCD_B_BYTES = 8 * 128 * 2;        // one site's B tile: 8 rows x 128 K
constexpr uint32_t TCD_WAIT = 1u << 22;         // bounded mbarrier polls (a round takes microseconds)
constexpr int TCD_THREADS = 128;

struct TcdArgs {
  Geom g;
  const char* links;  // 16-bit link storage (16 blocks)
  size_t blk_bytes;
  int out_parity;
  unsigned* out;      // [cb][color][nrhs] words (re, im)
  const unsigned* in;
  int nrhs;           // vectors per site, <= 64
  int* err;
};

inline size_t tcd_smem_bytes() {
  return (size_t)TCD_SITES * (TCD_A_BYTES + TCD_B_BYTES) + TCD_SITES * 16 * sizeof(int) + 64;
}

// Row n of hop h's B core matrix (8 halves = 4 words) for output real n = 2 i + part.
// Forward:  out_i += W v:       re row (W_ij) with im negated, im row (W_ij) halves swapped.
// Backward: out_i -= W_ji^* v:  re row -(W_ji) both halves, im row (W_ji) swapped, high half negated.
__device__ __forceinline__ unsigned swap_halves(unsigned w) { return __byte_perm(w, 0u, 0x1032); }

template <typename H>
__global__ void __launch_bounds__(TCD_THREADS) dslash_tc_kernel(const TcdArgs k) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem;
  unsigned char* Bt = smem + TCD_SITES * TCD_A_BYTES;
  int* nbtab = reinterpret_cast<int*>(Bt + TCD_SITES * TCD_B_BYTES);  // [site][hop]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(nbtab + TCD_SITES * 16);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Geom& g = k.g;
  const int p = k.out_parity, n = k.nrhs;

  // rows beyond nrhs and the two padding columns of every hop stay zero (finite) for the whole run
  for (int i = tid; i < TCD_SITES * (TCD_A_BYTES + TCD_B_BYTES) / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) tc::mbar_init(tc::smem_addr(mbar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = std::is_same<H, __half>::value ? tc::idesc_f16_f32(64, 8) : tc::idesc_bf16_f32(64, 8);
  const int rounds = (g.half + TCD_SITES - 1) / TCD_SITES;
  uint32_t phase = 0;
  bool failed = false;

  for (int round = blockIdx.x; round < rounds && !failed; round += gridDim.x) {
    const int cb0 = round * TCD_SITES;
    // neighbour of every (site, hop)
    if (tid < TCD_SITES * 16) {
      const int s = tid >> 4, h = tid & 15;
      const int cb = cb0 + s;
      int nb = -1;
      if (cb < g.half) {
        int c[4];
        site_coords(g, p, cb, c);
        const int idx = lex_index(g, c);
        const int mu = h >> 2, kind = (h >> 1) & 1;
        nb = neighbour_cb(g, c, idx, mu, (h & 1) ? (kind ? -3 : -1) : (kind ? 3 : 1));
      }
      nbtab[tid] = nb;
    }
    __syncthreads();
    // A rows: asynchronous 4-byte copies straight into the K-major rows (no register staging, every
    // copy of the round in flight at once); thread m = tid % 64 takes every other (site, hop)
    {
      const int m = tid & 63;
      if (m < n) {
#pragma unroll 4
        for (int sh = tid >> 6; sh < TCD_SITES * 16; sh += 2) {
          const int nb = nbtab[sh];
          if (nb < 0) continue;
          const uint32_t dst =
              tc::smem_addr(A + (sh >> 4) * TCD_A_BYTES + (m >> 3) * 2048 + (sh & 15) * 128 + (m & 7) * 16);
          const unsigned* src = k.in + (size_t)nb * 3 * n + m;
#pragma unroll
          for (int c = 0; c < 3; ++c)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 4 * c), "l"(src + (size_t)c * n)
                         : "memory");
        }
      }
    }
    // B: each (site, hop)'s link in real form, while the copies are in flight (one thread each)
    if (tid < TCD_SITES * 16 && nbtab[tid] >= 0) {
      const int s = tid >> 4, h = tid & 15;
      const int mu = h >> 2, kind = (h >> 1) & 1;
      const bool back = h & 1;
      // the hop's link as stored: entries 0-7 in two 16-byte words, entry 8 in a 4-byte word
      const char* blk = k.links + (size_t)(((back ? 1 - p : p) * 2 + kind) * 4 + mu) * k.blk_bytes;
      const int lcb = back ? nbtab[tid] : cb0 + s;
      const uint4 w0 = ld_stream(reinterpret_cast<const uint4*>(blk) + lcb);
      const uint4 w1 = ld_stream(reinterpret_cast<const uint4*>(blk) + (size_t)g.half + lcb);
      const unsigned w8 = ld_stream(reinterpret_cast<const unsigned*>(blk + (size_t)32 * g.half) + lcb);
      const unsigned W[9] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w8};
      unsigned char* brow = Bt + s * TCD_B_BYTES + h * 128;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        uint4 re, im;
        if (!back) {
          re = make_uint4(W[3 * i] ^ 0x80000000u, W[3 * i + 1] ^ 0x80000000u, W[3 * i + 2] ^ 0x80000000u, 0u);
          im = make_uint4(swap_halves(W[3 * i]), swap_halves(W[3 * i + 1]), swap_halves(W[3 * i + 2]), 0u);
        } else {
          re = make_uint4(W[i] ^ 0x80008000u, W[3 + i] ^ 0x80008000u, W[6 + i] ^ 0x80008000u, 0u);
          im = make_uint4(swap_halves(W[i]) ^ 0x80000000u, swap_halves(W[3 + i]) ^ 0x80000000u,
                          swap_halves(W[6 + i]) ^ 0x80000000u, 0u);
        }
        *reinterpret_cast<uint4*>(brow + (2 * i) * 16) = re;
        *reinterpret_cast<uint4*>(brow + (2 * i + 1) * 16) = im;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      // K-step-major order: consecutive MMAs accumulate into different sites' tiles, so the tensor core
      // is not held up by one tile's chain of accumulations
#pragma unroll 1
      for (int ks = 0; ks < 8; ++ks)
#pragma unroll
        for (int s = 0; s < TCD_SITES; ++s) {
          const uint32_t a0 = tc::smem_addr(A + s * TCD_A_BYTES), b0 = tc::smem_addr(Bt + s * TCD_B_BYTES);
          tc::mma_bf16(tmem + s * 8, tc::desc_kmajor(a0 + ks * 256, 128), tc::desc_kmajor(b0 + ks * 256, 128), idesc,
                       ks > 0 ? 1u : 0u);
        }
      tc::commit(tc::smem_addr(mbar));
    }
    // one warp polls the mbarrier (bounded); the others wait at the block barrier without issuing
    const bool ok = warp == 0 ? tc::mbar_wait(tc::smem_addr(mbar), phase, TCD_WAIT) : true;
    phase ^= 1;
    if (__syncthreads_or(!ok)) failed = true;
    tc::fence_after_sync();
    // read back: warp w holds vectors 16 w .. 16 w + 15 in its lanes 0-15
    const int m = 16 * warp + lane;
#pragma unroll
    for (int s2 = 0; s2 < TCD_SITES; s2 += 2) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + s2 * 8, v);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int cb = cb0 + s2 + t;
        if (lane < 16 && m < n && cb < g.half) {
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const float re = failed ? __int_as_float(0x7fc00000) : v[8 * t + 2 * i];
            const float im = failed ? __int_as_float(0x7fc00000) : v[8 * t + 2 * i + 1];
            unsigned w;
            if constexpr (std::is_same<H, __half>::value) {
              __half2 hw = __floats2half2_rn(re, im);
              w = *reinterpret_cast<unsigned*>(&hw);
            } else {
              __nv_bfloat162 hw = __floats2bfloat162_rn(re, im);
              w = *reinterpret_cast<unsigned*>(&hw);
            }
            k.out[((size_t)cb * 3 + i) * n + m] = w;
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // the next round overwrites A and B, and the accumulators
  }
  if (failed) {
    if (tid == 0) atomicExch(k.err, 1);
    if (warp == 0) tc::mbar_wait(tc::smem_addr(mbar), phase ^ 1, TCD_WAIT);  // let the outstanding MMAs drain
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 32);
}

// D on interleaved 16-bit vectors with the tensor cores: c.nrhs <= 64 vectors per site (a multiple of 4),
// plain epilogue. err: a device flag set when a bounded wait ran out.
int dslash_tc_launch(hisq_ctx* ctx, int prec, const DslashCall& c, int* err) {
  if (prec != HISQ_F16 && prec != HISQ_BF16) return set_error(HISQ_EINVAL, "tensor-core Dslash: 16-bit storage only");
  if (c.epi != EPI_PLAIN || !c.interleaved || c.nrhs < 4 || c.nrhs > 64 || c.nrhs % 4)
    return set_error(HISQ_EINVAL, "tensor-core Dslash: interleaved plain Dslash of 4..64 vectors");
  TcdArgs a;
  a.g = ctx->g;
  a.links = ctx->links[prec];
  a.blk_bytes = link_block_bytes(prec, ctx->g.half);
  a.out_parity = c.out_parity;
  a.out = (unsigned*)c.out;
  a.in = (const unsigned*)c.in;
  a.nrhs = c.nrhs;
  a.err = err;
  const size_t smem = tcd_smem_bytes();
  auto kern = prec == HISQ_F16 ? dslash_tc_kernel<__half> : dslash_tc_kernel<__nv_bfloat16>;
  if (!ctx->capturing) HISQ_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)smem));
  const int rounds = (ctx->g.half + TCD_SITES - 1) / TCD_SITES;
  int grid = ctx->num_sms * 3;  // three CTAs per SM: 3 x 73 KB of shared memory, 3 x 32 TMEM columns
  if (grid > rounds) grid = rounds;
  kern<<<grid, TCD_THREADS, smem, ctx->stream>>>(a);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  return HISQ_OK;
}

}  // namespace hisq
