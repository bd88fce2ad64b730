// Gauge-equivariant parallel-transport convolution (PTC) network on the GPU: forward layers,
// backward (input and weight gradients), Adam, and the preconditioner apply z = N(r).
//
// Layer: psi'_a(x) = sum_b sum_h W[a,b,h] (T_h psi_b)(x), 9 hops h = 0, +x..+t, -x..-t, with
//   T_+mu psi(x) = F_mu(x) psi(x+mu),  T_-mu psi(x) = F_mu(x-mu)^dag psi(x-mu)
// through the folded FP32 fat links of the context (the same links the Dslash uses).
// Network: layer 1 (1 -> C channels, full lattice), layer 2 (C -> 1, even sites); its input is an
// even-site vector embedded with zeros on odd sites.
//
// Work split: the parallel transport (3x3 link times colour vector) runs on CUDA cores; the
// channel mixing -- per colour, a [128 sites x 2*9*Cin] x [2*9*Cin x 2*Cout] real contraction of
// the transported vectors with the complex weights written as 2x2 real blocks -- runs on the
// fifth-generation tensor cores: operands in BF16 staged in shared memory (K-major), FP32
// accumulators in TMEM, one thread issuing tcgen05.mma, completion through an mbarrier, results
// read back with tcgen05.ld. The weight gradient (a contraction over sites) runs the same way
// with the site index as K. Master weights and Adam moments are FP32.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "internal.cuh"
#include "pdl.cuh"
#include "trace.h"
#include "tc.cuh"

namespace hisq {

bool is_device_ptr(const void* p);
double dslash_bytes(const hisq_ctx* ctx, int lp, int sp, int nrhs);

constexpr int PTC_TILE = 128;            // sites per tile = MMA M
constexpr int NHOP = 9;
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // bounded mbarrier polls (an MMA tile takes microseconds)

struct PtcGeom {
  Geom g;
  const char* fat32;  // FP32 link storage (16 blocks), fat = kind 0
  size_t blk_bytes;
};

__device__ __forceinline__ int lex_of(const Geom& g, int x, int y, int z, int t) {
  return x + g.stride[1] * y + g.stride[2] * z + g.stride[3] * t;
}

// T_h psi at site idx (coordinates c) for one channel: psi full-lattice [V][3] float2.
__device__ __forceinline__ void transport(const PtcGeom& G, const float2* __restrict__ psi, const int c[4], int idx,
                                          int h, cplx<float> out[3]) {
  if (h == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 v = psi[(size_t)idx * 3 + k];
      out[k] = {v.x, v.y};
    }
    return;
  }
  const Geom& g = G.g;
  const int mu = (h - 1) & 3;
  const bool fwd = h <= 4;
  int cm = c[mu] + (fwd ? 1 : -1);
  int n = idx + (fwd ? g.stride[mu] : -g.stride[mu]);
  if (cm >= g.L[mu]) n -= g.L[mu] * g.stride[mu];
  if (cm < 0) n += g.L[mu] * g.stride[mu];
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  // forward: F_mu(x) from block (parity(x), fat, mu) at cb(x); backward: F_mu(x-mu) at cb(x-mu)
  const int lpar = fwd ? par : 1 - par;
  const int lcb = fwd ? (idx >> 1) : (n >> 1);
  const char* blk = G.fat32 + (size_t)(lpar * 8 + mu) * G.blk_bytes;
  cplx<float> U[9];
  LinkIO<float>::load(blk, g.half, lcb, U);
  cplx<float> v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float2 w = psi[(size_t)n * 3 + k];
    v[k] = {w.x, w.y};
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    out[i] = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (fwd) cmac(out[i], U[3 * i + j], v[j]);
      else cmac_conj(out[i], U[3 * j + i], v[j]);
    }
  }
}

// T_h psi_b at site idx for CIN channels at once: the link is loaded once per hop and the CIN
// neighbour vectors are loaded together (memory-level parallelism).
template <int CIN>
__device__ __forceinline__ void transport_multi(const PtcGeom& G, const float2* __restrict__ psi, const int c[4],
                                                int idx, int h, cplx<float> (&out)[CIN][3]) {
  const Geom& g = G.g;
  const size_t cstride = (size_t)g.V * 3;
  if (h == 0) {
#pragma unroll
    for (int b = 0; b < CIN; ++b)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 v = psi[b * cstride + (size_t)idx * 3 + k];
        out[b][k] = {v.x, v.y};
      }
    return;
  }
  const int mu = (h - 1) & 3;
  const bool fwd = h <= 4;
  const int cm = c[mu] + (fwd ? 1 : -1);
  int n = idx + (fwd ? g.stride[mu] : -g.stride[mu]);
  if (cm >= g.L[mu]) n -= g.L[mu] * g.stride[mu];
  if (cm < 0) n += g.L[mu] * g.stride[mu];
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int lpar = fwd ? par : 1 - par;
  const int lcb = fwd ? (idx >> 1) : (n >> 1);
  cplx<float> U[9];
  LinkIO<float>::load(G.fat32 + (size_t)(lpar * 8 + mu) * G.blk_bytes, g.half, lcb, U);
  float2 v[CIN][3];
#pragma unroll
  for (int b = 0; b < CIN; ++b)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[b][k] = psi[b * cstride + (size_t)n * 3 + k];
#pragma unroll
  for (int b = 0; b < CIN; ++b)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      cplx<float> a = {0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const cplx<float> w = {v[b][j].x, v[b][j].y};
        if (fwd) cmac(a, U[3 * i + j], w);
        else cmac_conj(a, U[3 * j + i], w);
      }
      out[b][i] = a;
    }
}

// A pair (re, im) of bf16 at columns (col, col+1), col even: one 4-byte store.
__device__ __forceinline__ void put_bf16x2(unsigned char* tile, int row, int col, int K2, float re, float im) {
  *reinterpret_cast<__nv_bfloat162*>(tile + tc::kmajor_offset(row, col, K2)) = __floats2bfloat162_rn(re, im);
}

// Site of output row `row` of tile `tile`: full lattice (lexicographic) or even sites (cb order).
__device__ __forceinline__ bool tile_site(const Geom& g, bool even_only, int tile, int row, int c[4], int* idx,
                                          int* out_index) {
  const int n = even_only ? g.half : g.V;
  const int i = tile * PTC_TILE + row;
  if (i >= n) return false;
  if (even_only) {
    site_coords(g, 0, i, c);
    *idx = lex_index(g, c);
  } else {
    c[0] = i % g.L[0];
    c[1] = (i / g.L[0]) % g.L[1];
    c[2] = (i / (g.L[0] * g.L[1])) % g.L[2];
    c[3] = i / (g.L[0] * g.L[1] * g.L[2]);
    *idx = i;
  }
  *out_index = i;
  return true;
}

__device__ __forceinline__ void put_bf16(unsigned char* tile, int row, int col, int K2, float v) {
  *reinterpret_cast<__nv_bfloat16*>(tile + tc::kmajor_offset(row, col, K2)) = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------ forward layer
// out_a(x) = sum_{b,h} W[a][b][h] T_h in_b (x). in: [CIN][V][3] float2 (full lattice);
// out: [COUT][n_out][3] float2 with n_out = V (full) or V/2 (even sites, cb order).
// W: [COUT][CIN][9] float2 (FP32 master weights, rounded to BF16 for the tensor cores).
// Feature order is hop-major, k = h * CIN + b: with CIN = 8 each hop fills exactly one 16-column
// MMA K-step, so the operand tile can be staged a few hops at a time (HPP hops per pass, all
// passes accumulating into the same TMEM tile), which keeps the shared-memory footprint small
// enough for several CTAs per SM to overlap their fill, MMA and read-out phases.
template <int CIN>
struct FwdShape {
  static constexpr int HPP = CIN == 8 ? 3 : NHOP;                        // hops per pass
  static constexpr int NPASS = (NHOP + HPP - 1) / HPP;
  static constexpr int K2A = ((2 * CIN * HPP + 15) / 16) * 16;           // A columns per pass
  static constexpr int K2B = CIN == 8 ? 2 * CIN * NHOP : K2A;            // B columns (all hops)
};

template <int CIN, int COUT, bool OUT_EVEN>
__global__ void __launch_bounds__(256) k_ptc_forward(const PtcGeom G, const float2* __restrict__ in,
                                                     float2* __restrict__ out, const float2* __restrict__ W,
                                                     int* err, const int* skip) {
  if (skip && *skip) return;  // a solver cycle that has already finished (uniform)
  using S = FwdShape<CIN>;
  constexpr int K2A = S::K2A, K2B = S::K2B, HPP = S::HPP, NPASS = S::NPASS;
  constexpr int N2 = ((2 * COUT + 15) / 16) * 16;
  constexpr int TM_COLS = (3 * N2 <= 32) ? 32 : (3 * N2 <= 64) ? 64 : (3 * N2 <= 128) ? 128 : 256;
  static_assert(CIN == 1 || CIN == 8, "layer shapes of the network");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem;                               // 3 colours x [128 x K2A] bf16
  unsigned char* B = smem + 3 * PTC_TILE * K2A * 2;      // [N2 x K2B] bf16
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B + N2 * K2B * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const Geom& g = G.g;

  for (int i = tid; i < (3 * PTC_TILE * K2A + N2 * K2B) / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  // B[n][k]: k = 2*(h*CIN + b) + {re, im}; n = 2a + {re, im}; complex weight as a 2x2 real block
  for (int i = tid; i < COUT * CIN * NHOP; i += blockDim.x) {
    const int a = i / (CIN * NHOP), b = (i / NHOP) % CIN, h = i % NHOP;  // W[a][b][h]
    const float2 w = W[i];
    const int k = h * CIN + b;
    put_bf16(B, 2 * a, 2 * k, K2B, w.x);
    put_bf16(B, 2 * a, 2 * k + 1, K2B, -w.y);
    put_bf16(B, 2 * a + 1, 2 * k, K2B, w.y);
    put_bf16(B, 2 * a + 1, 2 * k + 1, K2B, w.x);
  }
  if (tid == 0) tc::mbar_init(tc::smem_addr(mbar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), TM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc::idesc_bf16_f32(PTC_TILE, N2);
  const int n_out = OUT_EVEN ? g.half : g.V;
  const int ntiles = (n_out + PTC_TILE - 1) / PTC_TILE;
  uint32_t phase = 0;
  bool failed = false;

  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
#pragma unroll 1
    for (int pass = 0; pass < NPASS && !failed; ++pass) {
      const int h0 = pass * HPP;
      const int nh = (NHOP - h0) < HPP ? (NHOP - h0) : HPP;
      // fill this pass's hops: work item = (row, hop); consecutive threads take consecutive sites
      for (int item = tid; item < PTC_TILE * nh; item += blockDim.x) {
        const int row = item % PTC_TILE, hl = item / PTC_TILE, h = h0 + hl;
        int c[4], idx, oi;
        cplx<float> u[CIN][3];
        // layer 1 (CIN = 1) reads the network input, an even-site vector embedded with zeros on odd
        // sites: the identity hop of an odd site and the +-mu hops of an even site transport zeros,
        // so they load no link and no vector
        bool live = tile_site(g, OUT_EVEN, tile, row, c, &idx, &oi);
        if (CIN == 1 && live) live = (h == 0) == (((c[0] + c[1] + c[2] + c[3]) & 1) == 0);
        if (live) {
          transport_multi<CIN>(G, in, c, idx, h, u);
        } else {
#pragma unroll
          for (int b = 0; b < CIN; ++b)
#pragma unroll
            for (int k = 0; k < 3; ++k) u[b][k] = {0.f, 0.f};
        }
#pragma unroll
        for (int b = 0; b < CIN; ++b) {
          const int k = hl * CIN + b;
#pragma unroll
          for (int col = 0; col < 3; ++col)
            put_bf16x2(A + col * PTC_TILE * K2A * 2, row, 2 * k, K2A, u[b][col].re, u[b][col].im);
        }
      }
      tc::fence_smem_to_async();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        const int ksteps = CIN == 8 ? nh : K2A / 16;
#pragma unroll 1
        for (int col = 0; col < 3; ++col) {
          const uint32_t a0 = tc::smem_addr(A + col * PTC_TILE * K2A * 2), b0 = tc::smem_addr(B);
#pragma unroll 1
          for (int ks = 0; ks < ksteps; ++ks) {
            const int kb = CIN == 8 ? (h0 + ks) : ks;  // K-step of B (a hop for CIN = 8)
            tc::mma_bf16(tmem + col * N2, tc::desc_kmajor(a0 + ks * 256, K2A), tc::desc_kmajor(b0 + kb * 256, K2B),
                         idesc, (pass > 0 || ks > 0) ? 1u : 0u);
          }
        }
        tc::commit(tc::smem_addr(mbar));
      }
      // the next pass (or tile) overwrites A: wait until the tensor core has read it
      const bool ok = tc::mbar_wait(tc::smem_addr(mbar), phase, WAIT_LIMIT);
      phase ^= 1;
      if (__syncthreads_or(!ok)) failed = true;
      tc::fence_after_sync();
    }
    if (failed) break;
    // readout: warp w reads TMEM lanes 32*(w%4).. (rows) for colours w/4, w/4 + 2, ...
    {
      const int q = warp & 3, row = 32 * q + (tid & 31);
      int c[4], idx, oi;
      const bool valid = tile_site(g, OUT_EVEN, tile, row, c, &idx, &oi);
#pragma unroll 1
      for (int col = warp >> 2; col < 3; col += (int)(blockDim.x >> 7)) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + col * N2, v);
        if (valid) {
#pragma unroll
          for (int a = 0; a < COUT; ++a) out[((size_t)a * n_out + oi) * 3 + col] = make_float2(v[2 * a], v[2 * a + 1]);
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    tc::mbar_wait(tc::smem_addr(mbar), phase ^ 1, WAIT_LIMIT);  // let the outstanding MMA drain
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TM_COLS);
}

// ------------------------------------------------------------------ backward: mixing + gather
// m_{b,h}(x) = sum_a conj(W[a][b][h]) g_a(x) on tensor cores; g: [COUT][n_in][3] (full or even
// sites), m: [CIN*9][V][3] full lattice (zero where g has no site).
template <int CIN, int COUT, bool IN_EVEN>
__global__ void __launch_bounds__(128) k_ptc_bwd_mix(const PtcGeom G, const float2* __restrict__ gout,
                                                     float2* __restrict__ m, const float2* __restrict__ W, int* err) {
  constexpr int K2 = ((2 * COUT + 15) / 16) * 16;
  constexpr int N2 = ((2 * NHOP * CIN + 15) / 16) * 16;
  constexpr int TM_COLS = (3 * N2 <= 32) ? 32 : (3 * N2 <= 64) ? 64 : (3 * N2 <= 128) ? 128 : (3 * N2 <= 256) ? 256 : 512;
  static_assert(N2 <= 256, "MMA N limit");
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem;                          // 3 x [128 x K2]
  unsigned char* B = smem + 3 * PTC_TILE * K2 * 2;  // [N2 x K2]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B + N2 * K2 * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const Geom& g = G.g;
  for (int i = tid; i < (3 * PTC_TILE * K2 + N2 * K2) / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  for (int i = tid; i < COUT * CIN * NHOP; i += blockDim.x) {
    const int a = i / (CIN * NHOP), j = i % (CIN * NHOP);
    const float2 w = W[i];
    // m_r = sum_a (w_r g_r + w_i g_i), m_i = sum_a (w_r g_i - w_i g_r)
    put_bf16(B, 2 * j, 2 * a, K2, w.x);
    put_bf16(B, 2 * j, 2 * a + 1, K2, w.y);
    put_bf16(B, 2 * j + 1, 2 * a, K2, -w.y);
    put_bf16(B, 2 * j + 1, 2 * a + 1, K2, w.x);
  }
  if (tid == 0) tc::mbar_init(tc::smem_addr(mbar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), TM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc::idesc_bf16_f32(PTC_TILE, N2);
  const int n_in = IN_EVEN ? g.half : g.V;
  const int ntiles = (n_in + PTC_TILE - 1) / PTC_TILE;
  uint32_t phase = 0;
  bool failed = false;
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    int c[4], idx, ii;
    const bool valid = tile_site(g, IN_EVEN, tile, tid, c, &idx, &ii);
#pragma unroll
    for (int a = 0; a < COUT; ++a)
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        float2 v = valid ? gout[((size_t)a * n_in + ii) * 3 + col] : make_float2(0.f, 0.f);
        unsigned char* Ac = A + col * PTC_TILE * K2 * 2;
        put_bf16(Ac, tid, 2 * a, K2, v.x);
        put_bf16(Ac, tid, 2 * a + 1, K2, v.y);
      }
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll 1
      for (int col = 0; col < 3; ++col) {
        const uint32_t a0 = tc::smem_addr(A + col * PTC_TILE * K2 * 2), b0 = tc::smem_addr(B);
#pragma unroll 1
        for (int ks = 0; ks < K2 / 16; ++ks)
          tc::mma_bf16(tmem + col * N2, tc::desc_kmajor(a0 + ks * 256, K2), tc::desc_kmajor(b0 + ks * 256, K2), idesc,
                       ks > 0);
      }
      tc::commit(tc::smem_addr(mbar));
    }
    const bool ok = tc::mbar_wait(tc::smem_addr(mbar), phase, WAIT_LIMIT);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
#pragma unroll 1
    for (int col = 0; col < 3; ++col) {
#pragma unroll 1
      for (int c16 = 0; c16 < N2; c16 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + col * N2 + c16, v);
        if (valid) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int j = c16 / 2 + q;
            if (j < CIN * NHOP) m[((size_t)j * g.V + idx) * 3 + col] = make_float2(v[2 * q], v[2 * q + 1]);
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    tc::mbar_wait(tc::smem_addr(mbar), phase ^ 1, WAIT_LIMIT);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TM_COLS);
}

// g_in_b(x) = sum_h T_h^dag m_{b,h} (x): T_0^dag = 1, T_+mu^dag = T_-mu, T_-mu^dag = T_+mu.
template <int CIN>
__global__ void k_ptc_bwd_gather(const PtcGeom G, const float2* __restrict__ m, float2* __restrict__ gin) {
  const Geom& g = G.g;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
    int c[4];
    c[0] = idx % g.L[0];
    c[1] = (idx / g.L[0]) % g.L[1];
    c[2] = (idx / (g.L[0] * g.L[1])) % g.L[2];
    c[3] = idx / (g.L[0] * g.L[1] * g.L[2]);
    for (int b = 0; b < CIN; ++b) {
      cplx<float> acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      for (int h = 0; h < NHOP; ++h) {
        const int hadj = h == 0 ? 0 : (h <= 4 ? h + 4 : h - 4);
        cplx<float> u[3];
        transport(G, m + (size_t)(b * NHOP + h) * g.V * 3, c, idx, hadj, u);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          acc[k].re += u[k].re;
          acc[k].im += u[k].im;
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) gin[((size_t)b * g.V + idx) * 3 + k] = make_float2(acc[k].re, acc[k].im);
    }
  }
}

// ------------------------------------------------------------------ weight gradient
// D[j][n] = sum_{x,col} U[j][(x,col)] Gm[(x,col)][n] with rows j = 2*(b*9+h) + {re, im} of
// u = T_h in_b and columns n = 2a + {re, im} of g_a; K = sites x colours, tiles of WG_SITES.
// Per-CTA partial sums (FP32, TMEM) go to part[cta][256][16]; k_ptc_wgrad_final combines.
constexpr int WG_SITES = 64;
constexpr int WG_K = WG_SITES * 3;  // 192 = 12 MMA K-steps

template <int CIN, int COUT, bool G_EVEN>
__global__ void __launch_bounds__(128) k_ptc_wgrad(const PtcGeom G, const float2* __restrict__ in,
                                                   const float2* __restrict__ gout, float* __restrict__ part,
                                                   int* err) {
  constexpr int MROWS = 2 * NHOP * CIN;      // real feature rows
  constexpr int MT = (MROWS + 127) / 128;    // M tiles of 128
  constexpr int N2 = ((2 * COUT + 15) / 16) * 16;
  constexpr int TM_COLS = (MT * N2 <= 32) ? 32 : 64;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* A = smem;                          // MT x [128 x WG_K]
  unsigned char* B = smem + MT * 128 * WG_K * 2;    // [N2 x WG_K]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(B + N2 * WG_K * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const Geom& g = G.g;
  for (int i = tid; i < (MT * 128 * WG_K + N2 * WG_K) / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) tc::mbar_init(tc::smem_addr(mbar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), TM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc::idesc_bf16_f32(128, N2);
  const int n_g = G_EVEN ? g.half : g.V;
  const int ntiles = (n_g + WG_SITES - 1) / WG_SITES;
  uint32_t phase = 0;
  bool failed = false, first = true;
  for (int tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x) {
    // threads 0..63 fill site (tid) of the tile; 64..127 idle while filling
    if (tid < WG_SITES) {
      const int i = tile * WG_SITES + tid;
      int c[4], idx = 0;
      const bool valid = i < n_g;
      if (valid) {
        if (G_EVEN) {
          site_coords(g, 0, i, c);
          idx = lex_index(g, c);
        } else {
          idx = i;
          c[0] = i % g.L[0];
          c[1] = (i / g.L[0]) % g.L[1];
          c[2] = (i / (g.L[0] * g.L[1])) % g.L[2];
          c[3] = i / (g.L[0] * g.L[1] * g.L[2]);
        }
      }
      for (int b = 0; b < CIN; ++b)
        for (int h = 0; h < NHOP; ++h) {
          cplx<float> u[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
          if (valid) transport(G, in + (size_t)b * g.V * 3, c, idx, h, u);
          const int j = 2 * (b * NHOP + h);
#pragma unroll
          for (int col = 0; col < 3; ++col) {
            const int k = col * WG_SITES + tid;
            put_bf16(A + (j / 128) * 128 * WG_K * 2, j % 128, k, WG_K, u[col].re);
            put_bf16(A + ((j + 1) / 128) * 128 * WG_K * 2, (j + 1) % 128, k, WG_K, u[col].im);
          }
        }
      for (int a = 0; a < COUT; ++a)
#pragma unroll
        for (int col = 0; col < 3; ++col) {
          float2 v = valid ? gout[((size_t)a * n_g + i) * 3 + col] : make_float2(0.f, 0.f);
          const int k = col * WG_SITES + tid;
          put_bf16(B, 2 * a, k, WG_K, v.x);
          put_bf16(B, 2 * a + 1, k, WG_K, v.y);
        }
    }
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        const uint32_t a0 = tc::smem_addr(A + mt * 128 * WG_K * 2), b0 = tc::smem_addr(B);
#pragma unroll 1
        for (int ks = 0; ks < WG_K / 16; ++ks)
          tc::mma_bf16(tmem + mt * N2, tc::desc_kmajor(a0 + ks * 256, WG_K), tc::desc_kmajor(b0 + ks * 256, WG_K),
                       idesc, (first && ks == 0) ? 0u : 1u);
      }
      tc::commit(tc::smem_addr(mbar));
    }
    first = false;
    const bool ok = tc::mbar_wait(tc::smem_addr(mbar), phase, WAIT_LIMIT);
    phase ^= 1;
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    tc::mbar_wait(tc::smem_addr(mbar), phase ^ 1, WAIT_LIMIT);
  }
  tc::fence_after_sync();
  // this CTA's partial: rows 32*warp + lane of each M tile, N2 columns
#pragma unroll 1
  for (int mt = 0; mt < MT; ++mt) {
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + mt * N2, v);
    const int row = mt * 128 + tid;
    float* dst = part + ((size_t)blockIdx.x * 256 + row) * 16;
#pragma unroll
    for (int q = 0; q < 16; ++q) dst[q] = first ? 0.f : v[q];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TM_COLS);
}

// gW[a][b][h] = (D[2j][2a] + D[2j+1][2a+1]) + i (D[2j][2a+1] - D[2j+1][2a]), j = b*9+h, summed over
// CTA partials in fixed order; scaled by `scale`. Output float2 [COUT][CIN][9].
__global__ void k_ptc_wgrad_final(const float* __restrict__ part, int nparts, int cin, int cout, float scale,
                                  float2* __restrict__ gW) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cout * cin * NHOP) return;
  const int a = i / (cin * NHOP), j = i % (cin * NHOP);
  double rr = 0, ii = 0, ri = 0, ir = 0;
  for (int p = 0; p < nparts; ++p) {
    const float* P = part + (size_t)p * 256 * 16;
    rr += P[(2 * j) * 16 + 2 * a];
    ii += P[(2 * j + 1) * 16 + 2 * a + 1];
    ri += P[(2 * j) * 16 + 2 * a + 1];
    ir += P[(2 * j + 1) * 16 + 2 * a];
  }
  gW[i] = make_float2((float)((rr + ii) * scale), (float)((ri - ir) * scale));
}

// ------------------------------------------------------------------ preconditioner apply (inference)
// The network is linear, so its two layers compose into one operator. With the input r on even sites
// (zeros on odd sites) and the output read on even sites x:
//   N(r)(x) = c0 r(x) + sum_{h != 0} T_h phi_h (x),   phi_h(y) = sum_{h' != 0} C[h][h'] (T_h' r)(y)
// on the odd sites y = x + h, with c0 = sum_a W2[a][0] W1[a][0] and C[h][h'] = sum_a W2[a][h] W1[a][h']
// (hops h, h' in +x..+t, -x..-t; at an even site only the identity hop of layer 1 sees r, at an odd
// site only its eight neighbour hops). The 8-channel activation is thereby replaced by the eight
// mixed transports phi_h of each odd site, written once and read once (an activation of half the
// lattice that layer 2 needs at x + h only), and each stencil pass reads every fat link once. The
// weights enter rounded to BF16, as on the tensor-core path that training uses.
__device__ __forceinline__ cplx<float> bf16c(float2 w) {
  return {__bfloat162float(__float2bfloat16_rn(w.x)), __bfloat162float(__float2bfloat16_rn(w.y))};
}

// mix[0] = c0, mix[1 + 8 (h-1) + (h'-1)] = C[h][h'], from W1 [C][1][9] and W2 [1][C][9].
__global__ void k_ptc_mixing(const float2* __restrict__ w1, const float2* __restrict__ w2, int C, float2* mix) {
  const int t = threadIdx.x;
  if (t > 64) return;
  const int h = t == 0 ? 0 : 1 + (t - 1) / 8, hp = t == 0 ? 0 : 1 + (t - 1) % 8;
  cplx<float> s = {0.f, 0.f};
  for (int a = 0; a < C; ++a) cmac(s, bf16c(w2[a * NHOP + h]), bf16c(w1[a * NHOP + hp]));
  mix[t] = make_float2(s.re, s.im);
}

// The hop h = 1..8 from a site with coordinates c (lexicographic idx, parity par): neighbour cb, and
// the link block and cb of the transport's link (F_mu(x) forward, F_mu(x - mu) backward).
__device__ __forceinline__ int ptc_hop(const PtcGeom& G, const int c[4], int idx, int par, int h, const char** blk,
                                       int* lcb) {
  const Geom& g = G.g;
  const int mu = (h - 1) & 3;
  const bool fwd = h <= 4;
  const int nb = neighbour_cb(g, c, idx, mu, fwd ? 1 : -1);
  *blk = G.fat32 + (size_t)((fwd ? par : 1 - par) * 8 + mu) * G.blk_bytes;
  *lcb = fwd ? (idx >> 1) : nb;
  return nb;
}

// Pass 1, odd sites y: phi_h(y) = sum_h' C[h][h'] (T_h' r)(y), stored as 8 planes [h-1][cb][3] of FP16
// pairs (relative rounding 2^-11, below the network's BF16 weights' 2^-8). Blocks of 128 held to 72
// registers (7 per SM): at 80 registers 32^3x8's 131,072 odd sites needed 1.12 waves of resident
// threads, and the second wave's few blocks ran alone (ncu: 41% of DRAM peak).
__global__ void __launch_bounds__(128, 7) k_ptc_apply_odd(const PtcGeom G, const float2* __restrict__ r,
                                                       __half2* __restrict__ phi, const float2* __restrict__ mix,
                                                       const int* skip) {
  griddep_wait();  // a programmatic dependent launch (pdl.cuh): nothing is touched before this
  griddep_launch_dependents();
  if (skip && *skip) return;
  const Geom& g = G.g;
  for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.half; cb += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, 1, cb, c);
    const int idx = lex_index(g, c);
    cplx<float> acc[8][3];
#pragma unroll
    for (int h = 0; h < 8; ++h)
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[h][k] = {0.f, 0.f};
#pragma unroll 1
    for (int hp = 1; hp <= 8; ++hp) {
      const char* blk;
      int lcb;
      const int nb = ptc_hop(G, c, idx, 1, hp, &blk, &lcb);
      cplx<float> U[9], v[3], s[3];
      LinkIO<float>::load(blk, g.half, lcb, U);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 w = __ldg(r + (size_t)nb * 3 + k);
        v[k] = {w.x, w.y};
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        s[i] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (hp <= 4) cmac(s[i], U[3 * i + j], v[j]);
          else cmac_conj(s[i], U[3 * j + i], v[j]);
        }
      }
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const float2 m = __ldg(mix + 1 + 8 * h + (hp - 1));
        const cplx<float> cm = {m.x, m.y};
#pragma unroll
        for (int k = 0; k < 3; ++k) cmac(acc[h][k], cm, s[k]);
      }
    }
#pragma unroll
    for (int h = 0; h < 8; ++h)
#pragma unroll
      for (int k = 0; k < 3; ++k) phi[((size_t)h * g.half + cb) * 3 + k] = __floats2half2_rn(acc[h][k].re, acc[h][k].im);
  }
}

// Pass 2, even sites x: z(x) = c0 r(x) + sum_h T_h phi_h (x).
__global__ void __launch_bounds__(256) k_ptc_apply_even(const PtcGeom G, const float2* __restrict__ r,
                                                        const __half2* __restrict__ phi, float2* __restrict__ z,
                                                        const float2* __restrict__ mix, const int* skip) {
  griddep_wait();  // a programmatic dependent launch (pdl.cuh): nothing is touched before this
  griddep_launch_dependents();
  if (skip && *skip) return;
  const Geom& g = G.g;
  const float2 m0 = __ldg(mix);
  const cplx<float> c0 = {m0.x, m0.y};
  for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.half; cb += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, 0, cb, c);
    const int idx = lex_index(g, c);
    cplx<float> acc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 w = __ldg(r + (size_t)cb * 3 + k);
      acc[k] = {0.f, 0.f};
      cmac(acc[k], c0, cplx<float>{w.x, w.y});
    }
#pragma unroll 4
    for (int h = 1; h <= 8; ++h) {
      const char* blk;
      int lcb;
      const int nb = ptc_hop(G, c, idx, 0, h, &blk, &lcb);
      cplx<float> U[9], v[3];
      LinkIO<float>::load(blk, g.half, lcb, U);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 w = __half22float2(__ldg(phi + ((size_t)(h - 1) * g.half + nb) * 3 + k));
        v[k] = {w.x, w.y};
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (h <= 4) cmac(acc[i], U[3 * i + j], v[j]);
          else cmac_conj(acc[i], U[3 * j + i], v[j]);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) z[(size_t)cb * 3 + k] = make_float2(acc[k].re, acc[k].im);
  }
}

// ------------------------------------------------------------------ small kernels
// Embed an even-site vector [half][3] into the full lattice (zeros on odd sites).
__global__ void k_embed_even(const Geom g, const float2* __restrict__ r, float2* __restrict__ full, const int* skip) {
  if (skip && *skip) return;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < g.V; idx += gridDim.x * blockDim.x) {
    const int x = idx % g.L[0], y = (idx / g.L[0]) % g.L[1], z = (idx / (g.L[0] * g.L[1])) % g.L[2],
              t = idx / (g.L[0] * g.L[1] * g.L[2]);
    const bool even = ((x + y + z + t) & 1) == 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) full[(size_t)idx * 3 + k] = even ? r[(size_t)(idx >> 1) * 3 + k] : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ int adj_hop(int h) { return h == 0 ? 0 : (h <= 4 ? h + 4 : h - 4); }

// Tied network: W2[0][a][h] = conj(W1[a][0][adj(h)]).
__global__ void k_tie(const float2* __restrict__ w1, float2* __restrict__ w2, int C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C * NHOP) return;
  const int a = i / NHOP, h = i % NHOP;
  const float2 w = w1[a * NHOP + adj_hop(h)];
  w2[i] = make_float2(w.x, -w.y);
}

// Tied gradient: G1[a][0][h] += conj(G2[0][a][adj(h)]).
__global__ void k_tie_grad(float2* __restrict__ g1, const float2* __restrict__ g2, int C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C * NHOP) return;
  const int a = i / NHOP, h = i % NHOP;
  const float2 g = g2[a * NHOP + adj_hop(h)];
  g1[i].x += g.x;
  g1[i].y -= g.y;
}

__global__ void k_accumulate(float* __restrict__ acc, const float* __restrict__ g, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) acc[i] += g[i];
}

// Adam on FP32 master weights with the real gradient 2*(Re G, Im G) of the Wirtinger gradient G.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ G,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gr = 2.f * G[i];
  m[i] = b1 * m[i] + (1.f - b1) * gr;
  v[i] = b2 * v[i] + (1.f - b2) * gr * gr;
  w[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

// ------------------------------------------------------------------ flexible CG
struct FcgState {
  double pq;             // <p, A p> (real: A Hermitian positive)
  double pr[2];          // <p, r>
  double qz[2];          // <q, z>
  double rr, rr_true, bb, tol2, scale;
  int done, iter, cycle_iter, cycle_limit, conv, nonfinite, breakdown, pad;
};

__device__ __forceinline__ void load3(const float2* v, size_t site, float2 o[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) o[k] = v[3 * site + k];
}

// alpha = <p, r> / <p, q>; e += alpha p; r -= alpha q; rr = |r|^2; inner convergence, cycle count.
__global__ void k_fcg_update(float2* __restrict__ e, float2* __restrict__ r, const float2* __restrict__ p,
                             const float2* __restrict__ q, int nsite, FcgState* st, double* partials,
                             unsigned* counter) {
  if (st->done) return;
  const double pq = st->pq;
  const bool ok = pq > 0.0 && isfinite(pq);
  const float ar = ok ? (float)(st->pr[0] / pq) : 0.f, ai = ok ? (float)(st->pr[1] / pq) : 0.f;
  double v = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsite; i += gridDim.x * blockDim.x) {
    float2 pv[3], qv[3], rv[3], ev[3];
    load3(p, i, pv);
    load3(q, i, qv);
    load3(r, i, rv);
    load3(e, i, ev);
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ev[k].x += ar * pv[k].x - ai * pv[k].y;
      ev[k].y += ar * pv[k].y + ai * pv[k].x;
      rv[k].x -= ar * qv[k].x - ai * qv[k].y;
      rv[k].y -= ar * qv[k].y + ai * qv[k].x;
      t += rv[k].x * rv[k].x + rv[k].y * rv[k].y;
      e[3 * (size_t)i + k] = ev[k];
      r[3 * (size_t)i + k] = rv[k];
    }
    v += (double)t;
  }
  __shared__ double red[32];
  const double s = block_sum_dyn(v, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (!last_block_done(counter)) return;
  const double tot = sum_partials_dyn(partials, gridDim.x, red);
  if (threadIdx.x != 0) return;
  st->rr = tot;
  if (!ok) st->breakdown = 1;
  if (!isfinite(tot)) st->nonfinite = 1;
  st->iter += 1;
  st->cycle_iter += 1;
  if (tot * st->scale * st->scale <= st->tol2 || st->cycle_iter >= st->cycle_limit || !ok || !isfinite(tot))
    st->done = 1;
}

// qz = <q, z> (complex, FP64 across sites)
__global__ void k_fcg_qz(const float2* __restrict__ q, const float2* __restrict__ z, int nsite, FcgState* st,
                         double* partials, unsigned* counter) {
  if (st->done) return;
  double vr = 0.0, vi = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsite; i += gridDim.x * blockDim.x) {
    float2 qv[3], zv[3];
    load3(q, i, qv);
    load3(z, i, zv);
    float tr = 0.f, ti = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      tr += qv[k].x * zv[k].x + qv[k].y * zv[k].y;
      ti += qv[k].x * zv[k].y - qv[k].y * zv[k].x;
    }
    vr += (double)tr;
    vi += (double)ti;
  }
  __shared__ double red[32];
  const double sr = block_sum_dyn(vr, red);
  const double si = block_sum_dyn(vi, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sr;
    partials[2 * blockIdx.x + 1] = si;
  }
  if (!last_block_done(counter)) return;
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a += __ldcg(partials + 2 * k);
    b += __ldcg(partials + 2 * k + 1);
  }
  a = block_sum_dyn(a, red);
  b = block_sum_dyn(b, red);
  if (threadIdx.x == 0) {
    st->qz[0] = a;
    st->qz[1] = b;
  }
}

// p = z + beta p with beta = -<q, z> / <p, q> (restart: beta = 0); pr = <p, r>.
__global__ void k_fcg_pupdate(float2* __restrict__ p, const float2* __restrict__ z, const float2* __restrict__ r,
                              int nsite, FcgState* st, int restart, double* partials, unsigned* counter) {
  if (st->done) return;
  const double pq = st->pq;
  const float br = restart ? 0.f : (float)(-st->qz[0] / pq), bi = restart ? 0.f : (float)(-st->qz[1] / pq);
  double vr = 0.0, vi = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsite; i += gridDim.x * blockDim.x) {
    float2 pv[3] = {}, zv[3], rv[3];
    if (!restart) load3(p, i, pv);  // a restart never reads p (it may hold stale data)
    load3(z, i, zv);
    load3(r, i, rv);
    float tr = 0.f, ti = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float nx = zv[k].x + br * pv[k].x - bi * pv[k].y;
      const float ny = zv[k].y + br * pv[k].y + bi * pv[k].x;
      p[3 * (size_t)i + k] = make_float2(nx, ny);
      tr += nx * rv[k].x + ny * rv[k].y;  // Re conj(p) r
      ti += nx * rv[k].y - ny * rv[k].x;  // Im conj(p) r
    }
    vr += (double)tr;
    vi += (double)ti;
  }
  __shared__ double red[32];
  const double sr = block_sum_dyn(vr, red);
  const double si = block_sum_dyn(vi, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sr;
    partials[2 * blockIdx.x + 1] = si;
  }
  if (!last_block_done(counter)) return;
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a += __ldcg(partials + 2 * k);
    b += __ldcg(partials + 2 * k + 1);
  }
  a = block_sum_dyn(a, red);
  b = block_sum_dyn(b, red);
  if (threadIdx.x == 0) {
    st->pr[0] = a;
    st->pr[1] = b;
  }
}

// Reliable update, part 1: x += scale e, e = 0 (FP64 x).
__global__ void k_fcg_fold(double2* __restrict__ x, float2* __restrict__ e, size_t n, const FcgState* st) {
  const double s = st->scale;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 ev = e[i];
    double2 xv = x[i];
    xv.x += s * (double)ev.x;
    xv.y += s * (double)ev.y;
    x[i] = xv;
    e[i] = make_float2(0.f, 0.f);
  }
}

// r_hi = b - A x (FP64): rr_true (and bb with init).
__global__ void k_fcg_residual(const double2* __restrict__ b, const double2* __restrict__ Ax, double2* __restrict__ rh,
                               size_t n, FcgState* st, int init, double* partials, unsigned* counter) {
  double v0 = 0.0, v1 = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 bv = b[i], av = Ax[i];
    const double2 rv = make_double2(bv.x - av.x, bv.y - av.y);
    rh[i] = rv;
    v0 += rv.x * rv.x + rv.y * rv.y;
    v1 += bv.x * bv.x + bv.y * bv.y;
  }
  __shared__ double red[32];
  const double s0 = block_sum_dyn(v0, red), s1 = block_sum_dyn(v1, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
  if (!last_block_done(counter)) return;
  double a = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    a += __ldcg(partials + 2 * k);
    c += __ldcg(partials + 2 * k + 1);
  }
  a = block_sum_dyn(a, red);
  c = block_sum_dyn(c, red);
  if (threadIdx.x == 0) {
    st->rr_true = a;
    if (init) st->bb = c;
    if (!isfinite(a)) st->nonfinite = 1;
  }
}

// Reliable update, part 2: converged? else r = r_hi / s, rr = |r|^2, new cycle (done = 0).
__global__ void k_fcg_reliable(const double2* __restrict__ rh, float2* __restrict__ r, size_t n, FcgState* st,
                               unsigned* counter) {
  const bool conv = st->rr_true <= st->tol2;
  const double s = sqrt(st->rr_true / (double)n);
  if (!conv && s > 0.0) {
    const double inv = 1.0 / s;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      const double2 w = rh[i];
      r[i] = make_float2((float)(w.x * inv), (float)(w.y * inv));
    }
  }
  if (last_block_done(counter) && threadIdx.x == 0) {
    st->conv = conv;
    st->done = conv ? 1 : 0;
    st->cycle_iter = 0;
    if (!conv && s > 0.0) {
      st->scale = s;
      st->rr = st->rr_true / (s * s);
    }
  }
}

}  // namespace hisq

// ------------------------------------------------------------------ flexible CG driver
namespace hisq {

static int fcg_true_residual(hisq_ctx* c, double2* x, const double2* b, double2* rh, double2* Ax, double2* t64,
                             FcgState* st, double a, int init, double* partials) {
  DslashCall c1;
  c1.out_parity = 1;
  c1.out = t64;
  c1.in = x;
  c1.nrhs = 1;
  c1.rhs_stride = c->g.half;
  int rc = dslash_launch(c, HISQ_F64, HISQ_F64, c1);
  if (rc != HISQ_OK) return rc;
  DslashCall c2 = c1;
  c2.out_parity = 0;
  c2.out = Ax;
  c2.in = t64;
  c2.y = x;
  c2.a = a;
  c2.epi = EPI_AXPY;
  if ((rc = dslash_launch(c, HISQ_F64, HISQ_F64, c2)) != HISQ_OK) return rc;
  const size_t n = (size_t)c->g.half * 3;
  k_fcg_residual<<<c->num_sms * 4, 256, 0, c->stream>>>(b, Ax, rh, n, st, init, partials, c->d_counters + 20);
  HISQ_CUDA(cudaGetLastError());
  note_launch(c);
  return HISQ_OK;
}

}  // namespace hisq

// ------------------------------------------------------------------ object + C ABI
struct hisq_ptc {
  hisq_ctx* ctx = nullptr;
  int C = 8;
  float2 *w1 = nullptr, *w2 = nullptr;  // FP32 master [C][1][9], [1][C][9]
  float *m1 = nullptr, *v1 = nullptr, *m2 = nullptr, *v2 = nullptr;
  float2 *g1 = nullptr, *g2 = nullptr;  // gradients
  int adam_t = 0;
  int tied = 0;  // layer 2 = adjoint of layer 1 (N = B^dag B)
  int* d_err = nullptr;
  float2* mix = nullptr;  // the composed network's mixing coefficients (65 complex), for the apply
};

namespace hisq {

static PtcGeom ptc_geom(const hisq_ctx* c) {
  PtcGeom G;
  G.g = c->g;
  G.fat32 = c->links[HISQ_F32];
  G.blk_bytes = link_block_bytes(HISQ_F32, c->g.half);
  return G;
}

template <int CIN, int COUT>
static size_t fwd_smem() {
  constexpr int N2 = ((2 * COUT + 15) / 16) * 16;
  return (size_t)3 * PTC_TILE * FwdShape<CIN>::K2A * 2 + (size_t)N2 * FwdShape<CIN>::K2B * 2 + 16;
}
template <int CIN, int COUT>
static size_t mix_smem() {
  constexpr int K2 = ((2 * COUT + 15) / 16) * 16, N2 = ((2 * NHOP * CIN + 15) / 16) * 16;
  return (size_t)3 * PTC_TILE * K2 * 2 + (size_t)N2 * K2 * 2 + 16;
}
template <int CIN, int COUT>
static size_t wg_smem() {
  constexpr int MT = (2 * NHOP * CIN + 127) / 128, N2 = ((2 * COUT + 15) / 16) * 16;
  return (size_t)MT * 128 * WG_K * 2 + (size_t)N2 * WG_K * 2 + 16;
}

// One persistent CTA per SM keeps TMEM demand (at most 512 columns) within one SM's TMEM.
template <typename K>
static int launch_tc(hisq_ctx* c, K kern, size_t smem, int nwork, const char* what) {
  // raise this kernel's dynamic shared-memory limit; inside the library's own stream capture the
  // same launch has already been made eagerly, so the attribute is set
  if (!c->capturing)
    HISQ_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int grid = c->num_sms;
  if (grid > nwork) grid = nwork;
  if (grid < 1) grid = 1;
  (void)what;
  return grid;
}

template <int CIN, int COUT, bool OUT_EVEN>
static int forward_layer(hisq_ptc* P, const float2* in, float2* out, const float2* W, const int* skip = nullptr) {
  hisq_ctx* c = P->ctx;
  auto kern = k_ptc_forward<CIN, COUT, OUT_EVEN>;
  const size_t smem = fwd_smem<CIN, COUT>() + 1024;
  const int n_out = OUT_EVEN ? c->g.half : c->g.V;
  int grid = launch_tc(c, kern, smem, (n_out + PTC_TILE - 1) / PTC_TILE, "ptc forward");
  if (grid < 0) return grid;
  // several CTAs per SM: as many as registers, shared memory and threads allow, and at most 6
  // (each holds 64 TMEM columns; 8 would fill the SM's 512)
  static int per_sm = 0;
  if (per_sm == 0 && !c->capturing) {
    cudaFuncAttributes fa;
    int dev = 0, smem_sm = 0;
    HISQ_CUDA(cudaFuncGetAttributes(&fa, (const void*)kern));
    HISQ_CUDA(cudaGetDevice(&dev));
    HISQ_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int by_regs = 65536 / ((fa.numRegs > 0 ? fa.numRegs : 64) * 256);
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    per_sm = by_regs < by_smem ? by_regs : by_smem;
    if (per_sm > 6) per_sm = 6;
    if (per_sm < 1) per_sm = 1;
  }
  const int ntiles = (n_out + PTC_TILE - 1) / PTC_TILE;
  grid = c->num_sms * (per_sm > 0 ? per_sm : 1);
  if (grid > ntiles) grid = ntiles;
  kern<<<grid, 256, smem, c->stream>>>(ptc_geom(c), in, out, W, P->d_err, skip);
  HISQ_CUDA(cudaGetLastError());
  note_launch(c);
  return HISQ_OK;
}

// z = N(r) for nvec even-site FP32 vectors (device), using workspaces of the context: the composed
// linear operator (mixing coefficients formed whenever the weights change, then one stencil pass over
// odd and one over even sites); phi needs 8 * V/2 * 3 half2 of workspace.
static int network_apply(hisq_ptc* P, float2* z, const float2* r, int nvec, __half2* phi, const int* skip = nullptr) {
  hisq_ctx* c = P->ctx;
  const size_t nh = (size_t)c->g.half * 3;
  const PtcGeom G = ptc_geom(c);
  // one site per thread (the grid-stride loops then run once); the block scheduler balances the waves
  const int grid_odd = (c->g.half + 127) / 128, grid_even = (c->g.half + 255) / 256;
  for (int v = 0; v < nvec; ++v) {
    const float2* rv = r + v * nh;
    float2* zv = z + v * nh;
    const float2* mix = P->mix;
    HISQ_CUDA(launch_dependent(c, k_ptc_apply_odd, grid_odd, 128, G, rv, phi, mix, skip));
    HISQ_CUDA(launch_dependent(c, k_ptc_apply_even, grid_even, 256, G, rv, (const __half2*)phi, zv, mix, skip));
    note_launch(c, 2);
  }
  return HISQ_OK;
}

static int check_err(hisq_ptc* P) {
  int e = 0;
  HISQ_CUDA(cudaMemcpyAsync(&e, P->d_err, sizeof(int), cudaMemcpyDeviceToHost, P->ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(P->ctx->stream));
  if (e) {
    cudaMemsetAsync(P->d_err, 0, sizeof(int), P->ctx->stream);
    return set_error(HISQ_ETIMEOUT, "a tensor-core completion wait ran out");
  }
  return HISQ_OK;
}

template <int CIN, int COUT, bool G_EVEN>
static int weight_grad(hisq_ptc* P, const float2* in, const float2* gout, float2* gW, float scale, float* part) {
  hisq_ctx* c = P->ctx;
  auto kern = k_ptc_wgrad<CIN, COUT, G_EVEN>;
  const size_t smem = wg_smem<CIN, COUT>() + 1024;
  const int n_g = G_EVEN ? c->g.half : c->g.V;
  int grid = launch_tc(c, kern, smem, (n_g + WG_SITES - 1) / WG_SITES, "ptc wgrad");
  if (grid < 0) return grid;
  kern<<<grid, 128, smem, c->stream>>>(ptc_geom(c), in, gout, part, P->d_err);
  HISQ_CUDA(cudaGetLastError());
  k_ptc_wgrad_final<<<1, 128, 0, c->stream>>>(part, grid, CIN, COUT, scale, gW);
  HISQ_CUDA(cudaGetLastError());
  note_launch(c, 2);
  return HISQ_OK;
}

template <int CIN, int COUT, bool IN_EVEN>
static int input_grad(hisq_ptc* P, const float2* gout, float2* m, float2* gin, const float2* W) {
  hisq_ctx* c = P->ctx;
  auto kern = k_ptc_bwd_mix<CIN, COUT, IN_EVEN>;
  const size_t smem = mix_smem<CIN, COUT>() + 1024;
  const int n_in = IN_EVEN ? c->g.half : c->g.V;
  int grid = launch_tc(c, kern, smem, (n_in + PTC_TILE - 1) / PTC_TILE, "ptc mix");
  if (grid < 0) return grid;
  HISQ_CUDA(cudaMemsetAsync(m, 0, (size_t)CIN * NHOP * c->g.V * 3 * sizeof(float2), c->stream));
  kern<<<grid, 128, smem, c->stream>>>(ptc_geom(c), gout, m, W, P->d_err);
  HISQ_CUDA(cudaGetLastError());
  k_ptc_bwd_gather<CIN><<<c->num_sms * 4, 128, 0, c->stream>>>(ptc_geom(c), m, gin);
  HISQ_CUDA(cudaGetLastError());
  note_launch(c, 2);
  return HISQ_OK;
}

// e = (N(b) - x) / |x|^2 / npairs on even sites, and the loss terms (host reduction of a copy).
__global__ void k_ptc_residual(const float2* __restrict__ z, const float2* __restrict__ x, float2* __restrict__ e,
                               size_t n, float inv_nx, double* __restrict__ partials) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 a = z[i], b = x[i];
    const float2 d = make_float2(a.x - b.x, a.y - b.y);
    e[i] = make_float2(d.x * inv_nx, d.y * inv_nx);
    s += (double)(d.x * d.x + d.y * d.y);
  }
  __shared__ double red[32];
  double t = block_sum_dyn(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void k_sum_sq(const float2* __restrict__ x, size_t n, double* __restrict__ partials) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2 a = x[i];
    s += (double)(a.x * a.x + a.y * a.y);
  }
  __shared__ double red[32];
  double t = block_sum_dyn(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

}  // namespace hisq

using namespace hisq;

extern "C" {

int hisq_ptc_create(hisq_ptc** out, hisq_ctx* ctx, int channels) {
  if (!out || !ctx) return set_error(HISQ_EINVAL, "null argument");
  if (channels != 8) return set_error(HISQ_EINVAL, "the PTC network has 8 hidden channels");
  if (!ctx->links[HISQ_F32]) return set_error(HISQ_EINVAL, "the PTC network needs FP32 links resident");
  hisq_ptc* P = new (std::nothrow) hisq_ptc();
  if (!P) return set_error(HISQ_ENOMEM, "host allocation");
  P->ctx = ctx;
  P->C = channels;
  const size_t nw = (size_t)channels * NHOP;
  cudaError_t e = cudaMalloc(&P->w1, nw * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&P->w2, nw * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&P->g1, nw * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&P->g2, nw * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&P->m1, 4 * nw * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(P->m1, 0, 4 * nw * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&P->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(P->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&P->mix, 65 * sizeof(float2));
  if (e != cudaSuccess) {
    hisq_ptc_destroy(P);
    return cuda_error(e, "ptc buffers");
  }
  P->v1 = P->m1 + nw * 2;
  P->m2 = P->v1 + nw * 2;
  P->v2 = P->m2 + nw * 2;
  *out = P;
  return HISQ_OK;
}

int hisq_ptc_destroy(hisq_ptc* P) {
  if (!P) return HISQ_OK;
  // the bound context may already be gone: touch only the network's own buffers (cudaFree
  // waits for the device work that may still use them)
  cudaFree(P->w1);
  cudaFree(P->w2);
  cudaFree(P->g1);
  cudaFree(P->g2);
  cudaFree(P->m1);
  cudaFree(P->d_err);
  cudaFree(P->mix);
  delete P;
  return HISQ_OK;
}

int hisq_ptc_set_weights(hisq_ptc* P, const float* w1, const float* w2) {
  if (!P || !w1 || !w2) return set_error(HISQ_EINVAL, "null argument");
  const size_t nb = (size_t)P->C * NHOP * sizeof(float2);
  HISQ_CUDA(cudaMemcpyAsync(P->w1, w1, nb, cudaMemcpyDefault, P->ctx->stream));
  HISQ_CUDA(cudaMemcpyAsync(P->w2, w2, nb, cudaMemcpyDefault, P->ctx->stream));
  HISQ_CUDA(cudaMemsetAsync(P->m1, 0, 4 * nb, P->ctx->stream));
  P->adam_t = 0;
  if (P->tied) k_tie<<<1, 128, 0, P->ctx->stream>>>(P->w1, P->w2, P->C);
  k_ptc_mixing<<<1, 96, 0, P->ctx->stream>>>(P->w1, P->w2, P->C, P->mix);
  HISQ_CUDA(cudaGetLastError());
  HISQ_CUDA(cudaStreamSynchronize(P->ctx->stream));
  return HISQ_OK;
}

int hisq_ptc_set_tied(hisq_ptc* P, int tied) {
  if (!P) return set_error(HISQ_EINVAL, "null network");
  P->tied = tied ? 1 : 0;
  if (P->tied) {
    k_tie<<<1, 128, 0, P->ctx->stream>>>(P->w1, P->w2, P->C);
    k_ptc_mixing<<<1, 96, 0, P->ctx->stream>>>(P->w1, P->w2, P->C, P->mix);
    HISQ_CUDA(cudaGetLastError());
    HISQ_CUDA(cudaStreamSynchronize(P->ctx->stream));
  }
  return HISQ_OK;
}

int hisq_ptc_bind(hisq_ptc* P, hisq_ctx* c) {
  if (!P || !c) return set_error(HISQ_EINVAL, "null argument");
  for (int m = 0; m < 4; ++m)
    if (c->g.L[m] != P->ctx->g.L[m]) return set_error(HISQ_EINVAL, "lattice shape differs");
  if (!c->links[HISQ_F32]) return set_error(HISQ_EINVAL, "the PTC network needs FP32 links resident");
  if (c->stream != P->ctx->stream) cudaStreamSynchronize(P->ctx->stream);
  P->ctx = c;
  return HISQ_OK;
}

int hisq_ptc_get_weights(hisq_ptc* P, float* w1, float* w2) {
  if (!P || !w1 || !w2) return set_error(HISQ_EINVAL, "null argument");
  const size_t nb = (size_t)P->C * NHOP * sizeof(float2);
  HISQ_CUDA(cudaMemcpyAsync(w1, P->w1, nb, cudaMemcpyDefault, P->ctx->stream));
  HISQ_CUDA(cudaMemcpyAsync(w2, P->w2, nb, cudaMemcpyDefault, P->ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(P->ctx->stream));
  return HISQ_OK;
}

int hisq_ptc_apply(hisq_ptc* P, float* z, const float* r, int nvec) {
  if (!P || !z || !r || nvec < 1) return set_error(HISQ_EINVAL, "bad argument");
  if (!P->ctx->links_ready) return set_error(HISQ_ENOLINKS, "links not loaded");
  if (!is_device_ptr(z) || !is_device_ptr(r)) return set_error(HISQ_EINVAL, "device vectors only");
  hisq_ctx* c = P->ctx;
  __half2* phi = (__half2*)workspace(c, "ptc_phi", (size_t)8 * c->g.half * 3 * sizeof(__half2));
  if (!phi) return set_error(HISQ_ENOMEM, "ptc workspace");
  // the composed apply has no tensor-core wait to report: asynchronous on the stream, like hisq_dslash
  return network_apply(P, (float2*)z, (const float2*)r, nvec, phi);
}

// Loss (mean over pairs of |N(b)-x|^2/|x|^2) and Wirtinger gradients of both layers for npairs
// even-site FP32 (b, x) pairs; with lr > 0 an Adam step follows. g1, g2, loss: optional host outputs.
int hisq_ptc_train_step(hisq_ptc* P, const float* b, const float* x, int npairs, float lr, float* loss_out,
                        float* g1_out, float* g2_out) {
  TraceRange trace("hisq_ptc_train_step");
  if (!P || !b || !x || npairs < 1) return set_error(HISQ_EINVAL, "bad argument");
  if (!P->ctx->links_ready) return set_error(HISQ_ENOLINKS, "links not loaded");
  if (!is_device_ptr(b) || !is_device_ptr(x)) return set_error(HISQ_EINVAL, "device vectors only");
  hisq_ctx* c = P->ctx;
  const int C = P->C;
  const size_t V3 = (size_t)c->g.V * 3, nh = (size_t)c->g.half * 3;
  float2* psi0 = (float2*)workspace(c, "ptc_psi0", V3 * sizeof(float2));
  float2* psi1 = (float2*)workspace(c, "ptc_psi1", (size_t)C * V3 * sizeof(float2));
  float2* z = (float2*)workspace(c, "ptc_z", nh * sizeof(float2));
  float2* e = (float2*)workspace(c, "ptc_e", nh * sizeof(float2));
  float2* m = (float2*)workspace(c, "ptc_m", (size_t)C * NHOP * V3 * sizeof(float2));
  float2* gpsi1 = (float2*)workspace(c, "ptc_gpsi1", (size_t)C * V3 * sizeof(float2));
  float2* gw = (float2*)workspace(c, "ptc_gw", 4 * (size_t)C * NHOP * sizeof(float2));
  float* part = (float*)workspace(c, "ptc_part", (size_t)c->num_sms * 256 * 16 * sizeof(float));
  double* red = (double*)workspace(c, "ptc_red", 2 * 1024 * sizeof(double));
  if (!psi0 || !psi1 || !z || !e || !m || !gpsi1 || !gw || !part || !red) return set_error(HISQ_ENOMEM, "workspace");
  float2* gw1 = gw;
  float2* gw2 = gw + C * NHOP;
  float2* acc1 = gw + 2 * C * NHOP;
  float2* acc2 = gw + 3 * C * NHOP;
  HISQ_CUDA(cudaMemsetAsync(acc1, 0, 2 * (size_t)C * NHOP * sizeof(float2), c->stream));
  std::vector<double> hred(1024);
  double loss = 0.0;
  for (int q = 0; q < npairs; ++q) {
    const float2* bq = (const float2*)b + q * nh;
    const float2* xq = (const float2*)x + q * nh;
    // |x|^2 (deterministic partials, summed on the host)
    const int rg = 512;
    k_sum_sq<<<rg, 256, 0, c->stream>>>(xq, nh, red);
    HISQ_CUDA(cudaMemcpyAsync(hred.data(), red, rg * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HISQ_CUDA(cudaStreamSynchronize(c->stream));
    double nx = 0;
    for (int i = 0; i < rg; ++i) nx += hred[i];
    // forward
    k_embed_even<<<c->num_sms * 4, 256, 0, c->stream>>>(c->g, bq, psi0, nullptr);
    int rc = forward_layer<1, 8, false>(P, psi0, psi1, P->w1);
    if (rc == HISQ_OK) rc = forward_layer<8, 1, true>(P, psi1, z, P->w2);
    if (rc != HISQ_OK) return rc;
    // e = (z - x) / (|x|^2 npairs): dLoss/d(conj z)
    k_ptc_residual<<<rg, 256, 0, c->stream>>>(z, xq, e, nh, (float)(1.0 / (nx * npairs)), red);
    HISQ_CUDA(cudaMemcpyAsync(hred.data(), red, rg * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    HISQ_CUDA(cudaStreamSynchronize(c->stream));
    double ee = 0;
    for (int i = 0; i < rg; ++i) ee += hred[i];
    loss += ee / nx / npairs;
    // backward: layer 2 weights and input gradient, then layer 1 weights
    if ((rc = weight_grad<8, 1, true>(P, psi1, e, gw2, 1.f, part)) != HISQ_OK) return rc;
    if ((rc = input_grad<8, 1, true>(P, e, m, gpsi1, P->w2)) != HISQ_OK) return rc;
    if ((rc = weight_grad<1, 8, false>(P, psi0, gpsi1, gw1, 1.f, part)) != HISQ_OK) return rc;
    note_launch(c, 4);
    // accumulate over pairs
    k_accumulate<<<1, 256, 0, c->stream>>>((float*)acc1, (const float*)gw1, 2 * C * NHOP);
    k_accumulate<<<1, 256, 0, c->stream>>>((float*)acc2, (const float*)gw2, 2 * C * NHOP);
    HISQ_CUDA(cudaGetLastError());
    note_launch(c, 2);
  }
  int rc = check_err(P);
  if (rc != HISQ_OK) return rc;
  if (P->tied) {
    k_tie_grad<<<1, 128, 0, c->stream>>>(acc1, acc2, C);
    HISQ_CUDA(cudaGetLastError());
    note_launch(c);
  }
  if (loss_out) *loss_out = (float)loss;
  if (g1_out) HISQ_CUDA(cudaMemcpy(g1_out, acc1, (size_t)C * NHOP * sizeof(float2), cudaMemcpyDeviceToHost));
  if (g2_out) HISQ_CUDA(cudaMemcpy(g2_out, acc2, (size_t)C * NHOP * sizeof(float2), cudaMemcpyDeviceToHost));
  if (lr > 0.f) {
    P->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)P->adam_t), c2 = 1.f - powf(b2, (float)P->adam_t);
    const int n = 2 * C * NHOP;
    k_adam<<<1, 256, 0, c->stream>>>((float*)P->w1, P->m1, P->v1, (const float*)acc1, n, lr, b1, b2, 1e-8f, c1, c2);
    if (P->tied)
      k_tie<<<1, 128, 0, c->stream>>>(P->w1, P->w2, C);
    else
      k_adam<<<1, 256, 0, c->stream>>>((float*)P->w2, P->m2, P->v2, (const float*)acc2, n, lr, b1, b2, 1e-8f, c1, c2);
    k_ptc_mixing<<<1, 96, 0, c->stream>>>(P->w1, P->w2, C, P->mix);
    HISQ_CUDA(cudaGetLastError());
    note_launch(c, 3);
    HISQ_CUDA(cudaStreamSynchronize(c->stream));
  }
  return HISQ_OK;
}


int hisq_fcg(hisq_ctx* c, hisq_ptc* P, double* x_user, const double* b_user, double mass, double rel_tol,
             int maxiter, const hisq_solver_opts* opts, hisq_solver_stats* stats) {
  TraceRange trace("hisq_fcg");
  if (!c || !P || !x_user || !b_user) return set_error(HISQ_EINVAL, "null argument");
  if (P->ctx != c) return set_error(HISQ_EINVAL, "the network belongs to another context");
  if (!c->links_ready) return set_error(HISQ_ENOLINKS, "links not loaded");
  if (!(mass > 0) || !(rel_tol > 0) || maxiter < 0) return set_error(HISQ_EINVAL, "need mass > 0, rel_tol > 0");
  if ((uintptr_t)x_user % 16 || (uintptr_t)b_user % 16) return set_error(HISQ_EINVAL, "vectors must be 16-byte aligned");
  hisq_solver_opts o;
  hisq_solver_opts_default(&o);
  if (opts) o = *opts;
  if (o.reliable_period < 1) return set_error(HISQ_EINVAL, "reliable_period must be >= 1");
  if (stats) memset(stats, 0, sizeof *stats);
  auto t_start = std::chrono::steady_clock::now();
  const long long l0 = c->launches;
  const int half = c->g.half;
  const size_t n = (size_t)half * 3;
  const bool xh = !is_device_ptr(x_user), bh = !is_device_ptr(b_user);
  double2* x = xh ? (double2*)workspace(c, "user_x", n * sizeof(double2)) : (double2*)x_user;
  double2* b = bh ? (double2*)workspace(c, "user_b", n * sizeof(double2)) : (double2*)b_user;
  double2* rh = (double2*)workspace(c, "fcg_rh", n * sizeof(double2));
  double2* Ax = (double2*)workspace(c, "fcg_Ax", n * sizeof(double2));
  double2* t64 = (double2*)workspace(c, "fcg_t64", n * sizeof(double2));
  float2* r = (float2*)workspace(c, "fcg_r", n * sizeof(float2));
  float2* p = (float2*)workspace(c, "fcg_p", n * sizeof(float2));
  float2* q = (float2*)workspace(c, "fcg_q", n * sizeof(float2));
  float2* t = (float2*)workspace(c, "fcg_t", n * sizeof(float2));
  float2* z = (float2*)workspace(c, "fcg_z", n * sizeof(float2));
  float2* e = (float2*)workspace(c, "fcg_e", n * sizeof(float2));
  __half2* phi = (__half2*)workspace(c, "ptc_phi", (size_t)8 * c->g.half * 3 * sizeof(__half2));
  FcgState* st = (FcgState*)workspace(c, "fcg_state", sizeof(FcgState));
  double* partials = (double*)workspace(c, "fcg_partials", 4 * (size_t)c->num_sms * 64 * sizeof(double));
  if (!x || !b || !rh || !Ax || !t64 || !r || !p || !q || !t || !z || !e || !phi || !st || !partials)
    return set_error(HISQ_ENOMEM, "fcg workspace");
  if (xh) HISQ_CUDA(cudaMemcpyAsync(x, x_user, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  if (bh) HISQ_CUDA(cudaMemcpyAsync(b, b_user, n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
  HISQ_CUDA(cudaMemsetAsync(e, 0, n * sizeof(float2), c->stream));
  FcgState* h = (FcgState*)c->pinned;
  memset(h, 0, sizeof(FcgState));
  h->scale = 1.0;
  h->cycle_limit = o.reliable_period;
  HISQ_CUDA(cudaMemcpyAsync(st, h, sizeof(FcgState), cudaMemcpyHostToDevice, c->stream));
  const double a = 4.0 * mass * mass;
  double* red = partials + 2 * (size_t)c->num_sms * 64;
  int rc = fcg_true_residual(c, x, b, rh, Ax, t64, st, a, 1, red);
  if (rc != HISQ_OK) return rc;
  HISQ_CUDA(cudaMemcpyAsync(h, st, sizeof(FcgState), cudaMemcpyDeviceToHost, c->stream));
  HISQ_CUDA(cudaStreamSynchronize(c->stream));
  if (!isfinite(h->bb) || !isfinite(h->rr_true)) return set_error(HISQ_ENONFINITE, "non-finite source or guess");
  h->tol2 = rel_tol * rel_tol * h->bb;
  HISQ_CUDA(cudaMemcpyAsync(&st->tol2, &h->tol2, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const int gb = c->num_sms * 4;
  auto restart = [&]() -> int {
    k_fcg_reliable<<<gb, 256, 0, c->stream>>>(rh, r, n, st, c->d_counters + 21);
    HISQ_CUDA(cudaGetLastError());
    int r2 = network_apply(P, z, r, 1, phi, &st->done);
    if (r2 != HISQ_OK) return r2;
    k_fcg_pupdate<<<gb, 256, 0, c->stream>>>(p, z, r, half, st, 1, red, c->d_counters + 22);
    HISQ_CUDA(cudaGetLastError());
    note_launch(c, 2);
    return HISQ_OK;
  };
  if ((rc = restart()) != HISQ_OK) return rc;
  // pre-tune the inner Dslash launches (idempotent) outside the capture
  DslashCall c1;
  c1.out_parity = 1;
  c1.out = t;
  c1.in = p;
  c1.nrhs = 1;
  c1.rhs_stride = half;
  DslashCall c2 = c1;
  c2.out_parity = 0;
  c2.out = q;
  c2.in = t;
  c2.y = p;
  c2.a = a;
  c2.epi = EPI_AXPY;
  c2.partials = partials;
  c2.dot_out = &st->pq;
  c2.counter = c->d_counters + 23;
  if ((rc = dslash_launch(c, HISQ_F32, HISQ_F32, c1)) != HISQ_OK) return rc;
  if ((rc = dslash_launch(c, HISQ_F32, HISQ_F32, c2)) != HISQ_OK) return rc;
  c1.skip = &st->done;
  c2.skip = &st->done;
  auto iteration = [&]() -> int {
    int r2 = dslash_launch(c, HISQ_F32, HISQ_F32, c1);
    if (r2 == HISQ_OK) r2 = dslash_launch(c, HISQ_F32, HISQ_F32, c2);
    if (r2 != HISQ_OK) return r2;
    k_fcg_update<<<gb, 256, 0, c->stream>>>(e, r, p, q, half, st, red, c->d_counters + 24);
    HISQ_CUDA(cudaGetLastError());
    if ((r2 = network_apply(P, z, r, 1, phi, &st->done)) != HISQ_OK) return r2;
    k_fcg_qz<<<gb, 256, 0, c->stream>>>(q, z, half, st, red, c->d_counters + 25);
    k_fcg_pupdate<<<gb, 256, 0, c->stream>>>(p, z, r, half, st, 0, red, c->d_counters + 22);
    HISQ_CUDA(cudaGetLastError());
    note_launch(c, 3);
    return HISQ_OK;
  };
  // one graph = one reliable cycle
  cudaGraph_t graph;
  cudaGraphExec_t exec = nullptr;
  HISQ_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  c->capturing = true;
  int crc = HISQ_OK;
  for (int i = 0; i < o.reliable_period && crc == HISQ_OK; ++i) crc = iteration();
  if (crc == HISQ_OK) {
    k_fcg_fold<<<gb, 256, 0, c->stream>>>(x, e, n, st);
    crc = fcg_true_residual(c, x, b, rh, Ax, t64, st, a, 0, red);
  }
  if (crc == HISQ_OK) crc = restart();
  c->capturing = false;
  cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
  if (crc != HISQ_OK) return crc;
  HISQ_CUDA(ce);
  size_t nodes = 0;
  cudaGraphGetNodes(graph, nullptr, &nodes);
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  HISQ_CUDA(ce);
  int status = HISQ_OK;
  int reliable = 0;
  HISQ_CUDA(cudaMemcpyAsync(h, st, sizeof(FcgState), cudaMemcpyDeviceToHost, c->stream));
  HISQ_CUDA(cudaStreamSynchronize(c->stream));
  while (!h->conv) {
    if (h->iter >= maxiter) {
      status = HISQ_ENOCONV;
      break;
    }
    HISQ_CUDA(cudaGraphLaunch(exec, c->stream));
    c->launches += (long long)nodes;
    ++reliable;
    HISQ_CUDA(cudaMemcpyAsync(h, st, sizeof(FcgState), cudaMemcpyDeviceToHost, c->stream));
    HISQ_CUDA(cudaStreamSynchronize(c->stream));
    if (h->nonfinite) {
      status = set_error(HISQ_ENONFINITE, "non-finite residual at iteration %d", h->iter);
      break;
    }
    if (h->breakdown) {
      status = set_error(HISQ_EBREAKDOWN, "<p, A p> <= 0 at iteration %d", h->iter);
      break;
    }
  }
  cudaGraphExecDestroy(exec);
  if ((rc = check_err(P)) != HISQ_OK) return rc;
  const double rel = h->bb > 0 ? sqrt(h->rr_true / h->bb) : sqrt(h->rr_true);
  if (stats) {
    stats->iters = h->iter;
    stats->reliable_updates = reliable;
    stats->converged = h->conv && status == HISQ_OK;
    stats->true_rel_residual = rel;
    stats->shift_residual[0] = rel;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    stats->dslash_calls = 2LL * h->iter + 2LL * (reliable + 1);
    stats->dslash_bytes = 2.0 * h->iter * dslash_bytes(c, HISQ_F32, HISQ_F32, 1) +
                          2.0 * (reliable + 1) * dslash_bytes(c, HISQ_F64, HISQ_F64, 1);
    stats->kernel_launches = c->launches - l0;
  }
  if (xh) {
    HISQ_CUDA(cudaMemcpyAsync(x_user, x, n * sizeof(double2), cudaMemcpyDeviceToHost, c->stream));
    HISQ_CUDA(cudaStreamSynchronize(c->stream));
  }
  if (status == HISQ_ENOCONV) return set_error(HISQ_ENOCONV, "fcg: no convergence in %d iterations (true residual %.3e)", h->iter, rel);
  return status;
}

}  // extern "C"
