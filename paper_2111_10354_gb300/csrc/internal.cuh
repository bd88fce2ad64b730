// Internal declarations of the HISQ GB300 library: context, precision traits, data
// layout in HBM, device helpers shared by the kernels.
//
// Layout in HBM (per resident precision R, real type of that precision):
//   links   one block per (parity p, kind k in {fat, long}, direction mu):
//           block(p,k,mu) holds the folded link of every site of parity p (numbered cb),
//           18 reals per link, split into "chunk planes" so that one thread loads one
//           link with a few 16-byte coalesced loads:
//             FP64      9 planes of double2          (1 complex entry each)
//             FP32      4 planes of float4 + 1 float2 (2 complex entries per float4)
//             FP16/BF16 2 planes of 16-byte vectors + 1 plane of 4 bytes (4 entries per 16 B)
//           plane j of block b starts at block base + (sum of earlier chunk sizes) * (V/2).
//   vectors the boundary layout [rhs][cb][color] of complex<R>, or the rhs-interleaved layout
//           [cb][color][rhs] of the interleaved entry points and of the mixed-precision solver's
//           multi-RHS inner vectors.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/hisq.h"
#include "df64.cuh"

namespace hisq {

// ------------------------------------------------------------------ complex arithmetic
template <typename T>
struct cplx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ void cmac(cplx<T>& acc, const cplx<T>& a, const cplx<T>& b) {  // acc += a*b
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// Double-float complex multiply-accumulate on lane pairs: (re, im) += (a.re, a.re) (b.re, b.im)
// + (-a.im, a.im) (b.im, b.re).
__device__ __forceinline__ void cmac(cplx<df64>& acc, const cplx<df64>& a, const cplx<df64>& b) {
  df64x2 c{make_float2(acc.re.hi, acc.im.hi), make_float2(acc.re.lo, acc.im.lo)};
  c = df2_fma({make_float2(a.re.hi, a.re.hi), make_float2(a.re.lo, a.re.lo)},
              {make_float2(b.re.hi, b.im.hi), make_float2(b.re.lo, b.im.lo)}, c);
  c = df2_fma({make_float2(-a.im.hi, a.im.hi), make_float2(-a.im.lo, a.im.lo)},
              {make_float2(b.im.hi, b.re.hi), make_float2(b.im.lo, b.re.lo)}, c);
  acc.re = df64(c.hi.x, c.lo.x);
  acc.im = df64(c.hi.y, c.lo.y);
}

template <typename T>
__device__ __forceinline__ void cmac_conj(cplx<T>& acc, const cplx<T>& a, const cplx<T>& b) {  // acc += conj(a)*b
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// ------------------------------------------------------------------ precision traits
template <typename R>
struct Real;
template <>
struct Real<double> {
  using acc = double;
  static constexpr int prec = HISQ_F64;
};
template <>
struct Real<float> {
  using acc = float;
  static constexpr int prec = HISQ_F32;
};
template <>
struct Real<__half> {
  using acc = float;
  static constexpr int prec = HISQ_F16;
};
template <>
struct Real<__nv_bfloat16> {
  using acc = float;
  static constexpr int prec = HISQ_BF16;
};
template <>
struct Real<df64> {
  using acc = df64;
  static constexpr int prec = HISQ_DF64;
};

constexpr int NPREC = 5;  // HISQ_F64 .. HISQ_DF64

// Bytes per real of a precision's storage (HISQ_DF64: two FP32 words per real).
__host__ __device__ inline size_t real_size(int prec) {
  return (prec == HISQ_F64 || prec == HISQ_DF64) ? 8 : prec == HISQ_F32 ? 4 : 2;
}

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];
  int stride[4];  // lexicographic strides 1, Lx, LxLy, LxLyLz
  int half_x;     // Lx / 2
  int half;       // V / 2 (sites per parity)
  int V;
};

// Coordinates of the site numbered cb among the sites of parity p.
__device__ __forceinline__ void site_coords(const Geom& g, int p, int cb, int c[4]) {
  int xh = cb % g.half_x;
  int rest = cb / g.half_x;
  c[1] = rest % g.L[1];
  rest /= g.L[1];
  c[2] = rest % g.L[2];
  c[3] = rest / g.L[2];
  c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
}

__device__ __forceinline__ int lex_index(const Geom& g, const int c[4]) {
  return c[0] + g.stride[1] * c[1] + g.stride[2] * c[2] + g.stride[3] * c[3];
}

// cb number of the neighbour of site (c, idx) at offset k (|k| < L) along mu.
__device__ __forceinline__ int neighbour_cb(const Geom& g, const int c[4], int idx, int mu, int k) {
  int cm = c[mu] + k;
  int n = idx + k * g.stride[mu];
  if (cm >= g.L[mu]) n -= g.L[mu] * g.stride[mu];
  if (cm < 0) n += g.L[mu] * g.stride[mu];
  return n >> 1;
}

// ------------------------------------------------------------------ link access
// Bytes of one link block (all sites of one parity, one kind, one direction).
__host__ __device__ inline size_t link_block_bytes(int prec, int half) { return (size_t)half * 18 * real_size(prec); }

// Link loads: read once per launch, so they bypass L1 and are first in line for L2 eviction
// (an evict-first L2 cache policy), which keeps the 16-fold reused input vector resident in L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ double2 ld_stream(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y)
               : "l"(p), "l"(l2_evict_first()));
  return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(l2_evict_first()));
  return v;
}
__device__ __forceinline__ float2 ld_stream(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(p), "l"(l2_evict_first()));
  return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(l2_evict_first()));
  return v;
}
__device__ __forceinline__ unsigned ld_stream(const unsigned* p) {
  unsigned v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(l2_evict_first()));
  return v;
}

template <typename R>
__device__ __forceinline__ cplx<float> unpack2(unsigned w);
template <>
__device__ __forceinline__ cplx<float> unpack2<__half>(unsigned w) {
  __half2 h = *reinterpret_cast<__half2*>(&w);
  float2 f = __half22float2(h);
  return {f.x, f.y};
}
template <>
__device__ __forceinline__ cplx<float> unpack2<__nv_bfloat16>(unsigned w) {
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&w);
  float2 f = __bfloat1622float2(h);
  return {f.x, f.y};
}

// Load the 3x3 link of site cb from a link block (row-major entries U[3*row+col]).
template <typename R>
struct LinkIO;

template <>
struct LinkIO<double> {
  __device__ __forceinline__ static void load(const char* blk, int half, int cb, cplx<double> U[9]) {
    const double2* p = reinterpret_cast<const double2*>(blk);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 v = ld_stream(p + (size_t)k * half + cb);
      U[k] = {v.x, v.y};
    }
  }
  __device__ __forceinline__ static void store(char* blk, int half, int cb, const cplx<double> U[9]) {
    double2* p = reinterpret_cast<double2*>(blk);
#pragma unroll
    for (int k = 0; k < 9; ++k) p[(size_t)k * half + cb] = make_double2(U[k].re, U[k].im);
  }
};

template <>
struct LinkIO<float> {
  __device__ __forceinline__ static void load(const char* blk, int half, int cb, cplx<float> U[9]) {
    const float4* p = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float4 v = ld_stream(p + (size_t)j * half + cb);
      U[2 * j] = {v.x, v.y};
      U[2 * j + 1] = {v.z, v.w};
    }
    const float2* q = reinterpret_cast<const float2*>(blk + (size_t)64 * half);
    float2 v = ld_stream(q + cb);
    U[8] = {v.x, v.y};
  }
  __device__ __forceinline__ static void store(char* blk, int half, int cb, const cplx<double> U[9]) {
    float4* p = reinterpret_cast<float4*>(blk);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      p[(size_t)j * half + cb] = make_float4((float)U[2 * j].re, (float)U[2 * j].im, (float)U[2 * j + 1].re,
                                             (float)U[2 * j + 1].im);
    float2* q = reinterpret_cast<float2*>(blk + (size_t)64 * half);
    q[cb] = make_float2((float)U[8].re, (float)U[8].im);
  }
};

// Double-float links: entry k of every site is one float4 (re.hi, re.lo, im.hi, im.lo) in plane k,
// 16 bytes like FP64. The split is round-to-nearest in both parts (|u - hi - lo| <= 2^-48 |u|).
template <>
struct LinkIO<df64> {
  __device__ __forceinline__ static void load(const char* blk, int half, int cb, cplx<df64> U[9]) {
    const float4* p = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 v = ld_stream(p + (size_t)k * half + cb);
      U[k] = {df64(v.x, v.y), df64(v.z, v.w)};
    }
  }
  __device__ __forceinline__ static void store(char* blk, int half, int cb, const cplx<double> U[9]) {
    float4* p = reinterpret_cast<float4*>(blk);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float rh = __double2float_rn(U[k].re), ih = __double2float_rn(U[k].im);
      p[(size_t)k * half + cb] = make_float4(rh, __double2float_rn(U[k].re - (double)rh), ih,
                                             __double2float_rn(U[k].im - (double)ih));
    }
  }
};

template <typename H>
struct LinkIO16 {
  __device__ __forceinline__ static void load(const char* blk, int half, int cb, cplx<float> U[9]) {
    const uint4* p = reinterpret_cast<const uint4*>(blk);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint4 v = ld_stream(p + (size_t)j * half + cb);
      U[4 * j + 0] = unpack2<H>(v.x);
      U[4 * j + 1] = unpack2<H>(v.y);
      U[4 * j + 2] = unpack2<H>(v.z);
      U[4 * j + 3] = unpack2<H>(v.w);
    }
    const unsigned* q = reinterpret_cast<const unsigned*>(blk + (size_t)32 * half);
    U[8] = unpack2<H>(ld_stream(q + cb));
  }
  __device__ __forceinline__ static unsigned pack(double re, double im);
  __device__ __forceinline__ static void store(char* blk, int half, int cb, const cplx<double> U[9]) {
    uint4* p = reinterpret_cast<uint4*>(blk);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint4 v;
      v.x = pack(U[4 * j].re, U[4 * j].im);
      v.y = pack(U[4 * j + 1].re, U[4 * j + 1].im);
      v.z = pack(U[4 * j + 2].re, U[4 * j + 2].im);
      v.w = pack(U[4 * j + 3].re, U[4 * j + 3].im);
      p[(size_t)j * half + cb] = v;
    }
    unsigned* q = reinterpret_cast<unsigned*>(blk + (size_t)32 * half);
    q[cb] = pack(U[8].re, U[8].im);
  }
};
template <>
__device__ __forceinline__ unsigned LinkIO16<__half>::pack(double re, double im) {
  // double -> half directly (one rounding), round to nearest even
  __half2 h = __halves2half2(__double2half(re), __double2half(im));
  return *reinterpret_cast<unsigned*>(&h);
}
template <>
__device__ __forceinline__ unsigned LinkIO16<__nv_bfloat16>::pack(double re, double im) {
  __nv_bfloat162 h = __halves2bfloat162(__double2bfloat16(re), __double2bfloat16(im));
  return *reinterpret_cast<unsigned*>(&h);
}
template <>
struct LinkIO<__half> : LinkIO16<__half> {};
template <>
struct LinkIO<__nv_bfloat16> : LinkIO16<__nv_bfloat16> {};

// ------------------------------------------------------------------ compressed long links
// A folded long link is c * V with V in SU(3) and c = naik * eta_mu(x) * (boundary sign), so its
// first two rows (12 reals) determine it: row2 = conj(row0 x row1) / c. Storage per block
// (parity, mu) of the low precisions: FP32 3 planes of float4 (entries 0-1, 2-3, 4-5);
// FP16/BF16 one 16-byte plane (entries 0-3) and one 8-byte plane (entries 4-5).
__host__ __device__ inline size_t long12_block_bytes(int prec, int half) { return (size_t)half * 12 * real_size(prec); }

template <typename T>
__device__ __forceinline__ void reconstruct_row2(cplx<T> U[9], T inv_c) {
  auto cross = [](const cplx<T>& a, const cplx<T>& b, const cplx<T>& c, const cplx<T>& d) {
    // conj(a*b - c*d)
    cplx<T> r;
    r.re = (a.re * b.re - a.im * b.im) - (c.re * d.re - c.im * d.im);
    r.im = -((a.re * b.im + a.im * b.re) - (c.re * d.im + c.im * d.re));
    return r;
  };
  cplx<T> r6 = cross(U[1], U[5], U[2], U[4]);
  cplx<T> r7 = cross(U[2], U[3], U[0], U[5]);
  cplx<T> r8 = cross(U[0], U[4], U[1], U[3]);
  U[6] = {r6.re * inv_c, r6.im * inv_c};
  U[7] = {r7.re * inv_c, r7.im * inv_c};
  U[8] = {r8.re * inv_c, r8.im * inv_c};
}

template <typename R>
struct Link12IO;
template <>
struct Link12IO<float> {
  __device__ __forceinline__ static void load(const char* blk, int half, int cb, cplx<float> U[9]) {
    const float4* p = reinterpret_cast<const float4*>(blk);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float4 v = ld_stream(p + (size_t)j * half + cb);
      U[2 * j] = {v.x, v.y};
      U[2 * j + 1] = {v.z, v.w};
    }
  }
  __device__ __forceinline__ static void store(char* blk, int half, int cb, const cplx<double> U[9]) {
    float4* p = reinterpret_cast<float4*>(blk);
#pragma unroll
    for (int j = 0; j < 3; ++j)
      p[(size_t)j * half + cb] = make_float4((float)U[2 * j].re, (float)U[2 * j].im, (float)U[2 * j + 1].re,
                                             (float)U[2 * j + 1].im);
  }
};
__device__ __forceinline__ uint2 ld_stream(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y)
               : "l"(p), "l"(l2_evict_first()));
  return v;
}
template <typename H>
struct Link12IO16 {
  __device__ __forceinline__ static void load(const char* blk, int half, int cb, cplx<float> U[9]) {
    uint4 v = ld_stream(reinterpret_cast<const uint4*>(blk) + cb);
    U[0] = unpack2<H>(v.x);
    U[1] = unpack2<H>(v.y);
    U[2] = unpack2<H>(v.z);
    U[3] = unpack2<H>(v.w);
    uint2 w = ld_stream(reinterpret_cast<const uint2*>(blk + (size_t)16 * half) + cb);
    U[4] = unpack2<H>(w.x);
    U[5] = unpack2<H>(w.y);
  }
  __device__ __forceinline__ static void store(char* blk, int half, int cb, const cplx<double> U[9]) {
    uint4 v;
    v.x = LinkIO16<H>::pack(U[0].re, U[0].im);
    v.y = LinkIO16<H>::pack(U[1].re, U[1].im);
    v.z = LinkIO16<H>::pack(U[2].re, U[2].im);
    v.w = LinkIO16<H>::pack(U[3].re, U[3].im);
    reinterpret_cast<uint4*>(blk)[cb] = v;
    uint2 w;
    w.x = LinkIO16<H>::pack(U[4].re, U[4].im);
    w.y = LinkIO16<H>::pack(U[5].re, U[5].im);
    reinterpret_cast<uint2*>(blk + (size_t)16 * half)[cb] = w;
  }
};
template <>
struct Link12IO<__half> : Link12IO16<__half> {};
template <>
struct Link12IO<__nv_bfloat16> : Link12IO16<__nv_bfloat16> {};

// Sign of a folded link from its site's coordinates: eta_mu(x) and, for a long link in t, the
// antiperiodic sign at t >= Lt-3.
__device__ __forceinline__ int folded_long_sign(const Geom& g, unsigned flags, int mu, int x0, int x1, int x2, int t) {
  int s = 1;
  if (flags & HISQ_APPLY_PHASES) {
    const int sum = (mu > 0 ? x0 : 0) + (mu > 1 ? x1 : 0) + (mu > 2 ? x2 : 0);
    if (sum & 1) s = -s;
  }
  if ((flags & HISQ_ANTIPERIODIC_T) && mu == 3 && t >= g.L[3] - 3) s = -s;
  return s;
}

// ------------------------------------------------------------------ vector access ([cb][3] complex<R>)
template <typename R>
struct VecIO;
template <>
struct VecIO<double> {
  __device__ __forceinline__ static void load(const void* v, size_t site, cplx<double> o[3]) {
    const double2* p = reinterpret_cast<const double2*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double2 w = p[c];
      o[c] = {w.x, w.y};
    }
  }
  __device__ __forceinline__ static void store(void* v, size_t site, const cplx<double> o[3]) {
    double2* p = reinterpret_cast<double2*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = make_double2(o[c].re, o[c].im);
  }
};
template <>
struct VecIO<float> {
  __device__ __forceinline__ static void load(const void* v, size_t site, cplx<float> o[3]) {
    const float2* p = reinterpret_cast<const float2*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 w = p[c];
      o[c] = {w.x, w.y};
    }
  }
  __device__ __forceinline__ static void store(void* v, size_t site, const cplx<float> o[3]) {
    float2* p = reinterpret_cast<float2*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = make_float2(o[c].re, o[c].im);
  }
};
template <>
struct VecIO<__half> {
  __device__ __forceinline__ static void load(const void* v, size_t site, cplx<float> o[3]) {
    const __half2* p = reinterpret_cast<const __half2*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 f = __half22float2(p[c]);
      o[c] = {f.x, f.y};
    }
  }
  __device__ __forceinline__ static void store(void* v, size_t site, const cplx<float> o[3]) {
    __half2* p = reinterpret_cast<__half2*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = __floats2half2_rn(o[c].re, o[c].im);
  }
};
template <>
struct VecIO<__nv_bfloat16> {
  __device__ __forceinline__ static void load(const void* v, size_t site, cplx<float> o[3]) {
    const __nv_bfloat162* p = reinterpret_cast<const __nv_bfloat162*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 f = __bfloat1622float2(p[c]);
      o[c] = {f.x, f.y};
    }
  }
  __device__ __forceinline__ static void store(void* v, size_t site, const cplx<float> o[3]) {
    __nv_bfloat162* p = reinterpret_cast<__nv_bfloat162*>(v) + 3 * site;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = __floats2bfloat162_rn(o[c].re, o[c].im);
  }
};

// ------------------------------------------------------------------ reductions
// Sum of a double over the block (blockDim.x a multiple of 32, <= 1024); thread 0 gets
// the result. Fixed order, so the sum is deterministic for a fixed launch shape.
__device__ __forceinline__ double block_sum_dyn(double v, double* smem /* 32 */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) smem[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) s += smem[k];
  }
  __syncthreads();
  return s;
}

// Marks this block done; returns true in every thread of the last block to finish.
// Partials written before the call are visible to the last block. The counter is
// reset by the last block so the next launch starts from zero.
__device__ __forceinline__ bool last_block_done(unsigned* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x * gridDim.y * gridDim.z - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return is_last;
}

// Deterministic sum of partials[0..n) by the (single) finishing block; thread 0 gets it.
// Eight independent accumulators per thread keep eight L2 loads in flight, so the single
// finishing block is not bound by a chain of dependent load latencies.
__device__ __forceinline__ double sum_partials_dyn(const double* partials, int n, double* smem) {
  double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int stride = blockDim.x;
  int i = threadIdx.x;
  for (; i + 7 * stride < n; i += 8 * stride) {
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] += __ldcg(partials + i + k * stride);
  }
  for (; i < n; i += stride) s[0] += __ldcg(partials + i);
  const double t = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
  return block_sum_dyn(t, smem);
}

}  // namespace hisq

// ------------------------------------------------------------------ context (host side)
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct hisq_ctx {
  hisq::Geom g;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  unsigned prec_mask = 0;
  char* links[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // per precision, 16 blocks each
  std::vector<unsigned char> t_loaded;                    // per t-slice
  unsigned load_flags = 0;
  bool links_ready = false;
  int num_sms = 0;
  int device = 0;                    // CUDA device current at hisq_create (where the links live)
  int autotune = 1;
  int pdl = 1;                       // Dslash launches as programmatic dependent launches
  std::map<std::string, DevBuf> ws;  // named device workspaces
  std::map<std::string, int> tune;   // kernel key -> block size
  void* pinned = nullptr;            // small pinned host buffer for scalar read-back
  unsigned* d_counters = nullptr;    // last-block counters (zeroed), 64 entries
  int* d_flag = nullptr;             // device error flag
  long long launches = 0;            // kernels executed (eager + graph nodes)
  double naik = 0.0;                 // != 0: long links also stored compressed (two rows), see below
  char* long12[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // per low precision, 8 blocks (parity, mu)
  bool capturing = false;            // inside this library's own stream capture
  // instantiated solver graphs, keyed by everything their kernels capture (buffers, shapes,
  // coefficients), so repeated solves replay them instead of capturing again
  std::map<std::string, std::pair<cudaGraphExec_t, long long>> graphs;
};

namespace hisq {

// Error state of the calling thread.
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
#define HISQ_CUDA(call)                                        \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return hisq::cuda_error(_e, #call); \
  } while (0)

void* workspace(hisq_ctx* ctx, const char* name, size_t bytes);  // nullptr on failure
void release_graphs(hisq_ctx* ctx);                               // destroy the cached solver graphs

// Count one eager kernel launch (launches recorded into a graph are counted per replay).
inline void note_launch(hisq_ctx* ctx, int n = 1) {
  if (!ctx->capturing) ctx->launches += n;
}

inline const char* link_block(const hisq_ctx* ctx, int prec, int parity, int kind, int mu) {
  return ctx->links[prec] + (size_t)((parity * 2 + kind) * 4 + mu) * link_block_bytes(prec, ctx->g.half);
}

// ------------------------------------------------------------------ Dslash launcher interface
// Epilogues of the Dslash kernel:
//   EPI_PLAIN   out = D in
//   EPI_AXPY    out = a * y - D in  and (optionally) dot[r] += Re<y_r, out_r> in FP64,
//               with a = 4 m^2 + sigma: the second half of A y = (4m^2+sigma) y - D_eo D_oe y.
enum { EPI_PLAIN = 0, EPI_AXPY = 1 };

struct DslashCall {
  int out_parity;
  void* out;
  const void* in;
  int nrhs;
  size_t rhs_stride;  // sites between consecutive rhs vectors (normally V/2)
  // EPI_AXPY
  const void* y = nullptr;
  double a = 0.0;
  const double* a_rhs = nullptr;  // host array [nrhs]: per-rhs coefficient (overrides a)
  double* partials = nullptr;  // [nrhs][grid] when non-null: reduce Re<y, out>
  double* dot_out = nullptr;   // [nrhs] final sums (written by the last block)
  unsigned* counter = nullptr;
  const int* skip = nullptr;  // device flag: skip the launch's work when set
  int epi = EPI_PLAIN;
  // vectors in the rhs-interleaved layout [cb][color][rhs] with nrhs vectors per site (one launch
  // for all of them; rhs_stride is unused), instead of [rhs][cb][color]
  bool interleaved = false;
};

// Launch D (link precision lp, spinor precision sp) on ctx->stream.
int dslash_launch(hisq_ctx* ctx, int lp, int sp, const DslashCall& call);
int dslash_grid(hisq_ctx* ctx, int lp, int sp, int nrhs, int epi, int* block_out);  // grid size used
double dslash_bytes(const hisq_ctx* ctx, int lp, int sp, int nrhs);

// Link packing (fold phases and boundary, convert to every resident precision).
int pack_links_slab(hisq_ctx* ctx, const double* d_fat, const double* d_long, int t0, int nt, unsigned flags);

}  // namespace hisq
