// Multi-RHS Dslash on the rhs-interleaved vector layout [cb][color][rhs] (the multi-RHS form of
// Sec. 3: one read of the links serves every vector of a site).
//
// With N vectors interleaved per site and colour, the N vectors of one neighbour are one contiguous
// block of 3 * N complex numbers, and each colour of it is a row of N. A thread owns "granules" of G
// vectors whose entries of one colour fill one 16-byte word: one FP64 vector, two FP32 vectors or four
// 16-bit vectors (N must be a multiple of G). TS threads share a site (TS a power of two, at most 32,
// so a site's threads sit in one warp) and own its granules in turn: thread sub owns granules sub,
// sub + TS, sub + 2 TS, ... So every vector load instruction reads, per site, TS consecutive 16-byte
// words of one colour row, and the TS threads of a site load the same link words in the same
// instruction: each link leaves HBM once per launch, each neighbour block is read coalesced.
#pragma once
#include <type_traits>

#include "dslash_impl.cuh"
#include "reduce_warp.cuh"

namespace hisq {

constexpr int MRHS_MAX = 64;

// Granule g of site `site` in a vector of ngr granules per colour row: word (site, colour c, g) of 16
// bytes holds the colour-c entries of vectors g*G .. g*G+G-1.
template <typename SR>
struct GranIO;
template <>
struct GranIO<double> {
  static constexpr int G = 1;
  __device__ __forceinline__ static size_t word(size_t site, int c, int ngr, int g) {
    return (site * 3 + c) * (size_t)ngr + g;
  }
  __device__ __forceinline__ static void load(const void* v, size_t site, int ngr, int g, cplx<double> o[1][3]) {
    const double2* p = reinterpret_cast<const double2*>(v);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 w = __ldg(p + word(site, c, ngr, g));
      o[0][c] = {w.x, w.y};
    }
  }
  __device__ __forceinline__ static void store(void* v, size_t site, int ngr, int g, const cplx<double> o[1][3]) {
    double2* p = reinterpret_cast<double2*>(v);
#pragma unroll
    for (int c = 0; c < 3; ++c) p[word(site, c, ngr, g)] = make_double2(o[0][c].re, o[0][c].im);
  }
};
template <>
struct GranIO<float> {
  static constexpr int G = 2;
  __device__ __forceinline__ static void load(const void* v, size_t site, int ngr, int g, cplx<float> o[2][3]) {
    const float4* p = reinterpret_cast<const float4*>(v);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float4 w = __ldg(p + (site * 3 + c) * (size_t)ngr + g);
      o[0][c] = {w.x, w.y};
      o[1][c] = {w.z, w.w};
    }
  }
  __device__ __forceinline__ static void store(void* v, size_t site, int ngr, int g, const cplx<float> o[2][3]) {
    float4* p = reinterpret_cast<float4*>(v);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      p[(site * 3 + c) * (size_t)ngr + g] = make_float4(o[0][c].re, o[0][c].im, o[1][c].re, o[1][c].im);
  }
};
template <typename H>
struct GranIO16 {
  static constexpr int G = 4;
  __device__ __forceinline__ static void load(const void* v, size_t site, int ngr, int g, cplx<float> o[4][3]) {
    const uint4* p = reinterpret_cast<const uint4*>(v);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint4 u = __ldg(p + (site * 3 + c) * (size_t)ngr + g);
      o[0][c] = unpack2<H>(u.x);
      o[1][c] = unpack2<H>(u.y);
      o[2][c] = unpack2<H>(u.z);
      o[3][c] = unpack2<H>(u.w);
    }
  }
  __device__ __forceinline__ static unsigned pack(const cplx<float>& z);
  __device__ __forceinline__ static void store(void* v, size_t site, int ngr, int g, const cplx<float> o[4][3]) {
    uint4* p = reinterpret_cast<uint4*>(v);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      p[(site * 3 + c) * (size_t)ngr + g] = make_uint4(pack(o[0][c]), pack(o[1][c]), pack(o[2][c]), pack(o[3][c]));
  }
};
template <>
__device__ __forceinline__ unsigned GranIO16<__half>::pack(const cplx<float>& z) {
  __half2 h = __floats2half2_rn(z.re, z.im);
  return *reinterpret_cast<unsigned*>(&h);
}
template <>
__device__ __forceinline__ unsigned GranIO16<__nv_bfloat16>::pack(const cplx<float>& z) {
  __nv_bfloat162 h = __floats2bfloat162_rn(z.re, z.im);
  return *reinterpret_cast<unsigned*>(&h);
}
template <>
struct GranIO<__half> : GranIO16<__half> {};
template <>
struct GranIO<__nv_bfloat16> : GranIO16<__nv_bfloat16> {};

struct MrhsArgs {
  Geom g;
  const char* links;  // resident link storage of the link precision (16 blocks)
  size_t blk_bytes;
  int out_parity;
  void* out;
  const void* in;
  int ngr;            // granules per site: N / G
  int ts;             // threads per site (power of two, <= 32)
  const void* y;      // EPI_AXPY
  double a[MRHS_MAX];  // per-rhs diagonal coefficient 4m^2 + sigma_r
  double* partials;   // [N][gridDim.x]
  double* dot_out;    // [N]
  unsigned* counter;
  const int* skip;
  const char* long12;
  size_t blk12;
  float inv_naik;
  unsigned flags;
};

// Register budget per form: the accumulators of NG * G vectors plus one link and one granule.
template <typename LR, int NV>
struct MrhsBounds {
  static constexpr int min_blocks = sizeof(LR) == 8 ? 1 : 2;
};

// One hop's link (uncompressed, or a compressed long link rebuilt from its two rows).
template <typename LR, bool COMP>
__device__ __forceinline__ void mrhs_link(const MrhsArgs& k, const char* blk, int lpar, int mu, int kind, int site,
                                          const int c[4], int yt, cplx<typename Real<LR>::acc> U[9]) {
  using A = typename Real<LR>::acc;
  if constexpr (COMP && sizeof(LR) < 8) {
    if (kind == 1) {
      Link12IO<LR>::load(k.long12 + (size_t)(lpar * 4 + mu) * k.blk12, k.g.half, site, U);
      const int sg = folded_long_sign(k.g, k.flags, mu, c[0], c[1], c[2], yt);
      reconstruct_row2(U, A(sg) * A(k.inv_naik));
      return;
    }
  }
  LinkIO<LR>::load(blk, k.g.half, site, U);
}

template <typename LR, typename SR, int NG, int EPI, bool COMP>
__global__ void __launch_bounds__(256, MrhsBounds<LR, NG * GranIO<SR>::G>::min_blocks)
    dslash_mrhs_kernel(const MrhsArgs k) {
  using A = typename Real<LR>::acc;
  using SA = typename Real<SR>::acc;
  using GIO = GranIO<SR>;
  constexpr int G = GIO::G;
  constexpr int NV = NG * G;  // vectors per thread
  if (k.skip && *k.skip) return;  // uniform over the grid
  const Geom& g = k.g;
  const int p = k.out_parity;
  const int ts = k.ts;
  const int sub = threadIdx.x & (ts - 1);
  // granule q of this thread is sub + q * ts; it exists while that is below ngr
  const int spb = blockDim.x / ts;
  const char* fwd = k.links + (size_t)(p * 8) * k.blk_bytes;
  const char* bwd = k.links + (size_t)((1 - p) * 8) * k.blk_bytes;
  double dot[NV];
#pragma unroll
  for (int r = 0; r < NV; ++r) dot[r] = 0.0;

  for (int cb = blockIdx.x * spb + (int)threadIdx.x / ts; cb < g.half; cb += gridDim.x * spb) {
    int c[4];
    site_coords(g, p, cb, c);
    const int idx = lex_index(g, c);
    cplx<A> acc[NV][3];
#pragma unroll
    for (int r = 0; r < NV; ++r)
#pragma unroll
      for (int i = 0; i < 3; ++i) acc[r][i] = {A(0), A(0)};

    // a rolled direction loop keeps the body of several vectors in the instruction cache
    constexpr int MU_UNROLL = (NV >= 4 || std::is_same<LR, df64>::value) ? 1 : 2;
#pragma unroll MU_UNROLL
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
      for (int kind = 0; kind < 2; ++kind) {
        const int hop = kind == 0 ? 1 : 3;
        // forward hop: + W_mu(x) in(x + hop mu)
        {
          const int nb = neighbour_cb(g, c, idx, mu, +hop);
          cplx<A> U[9];
          mrhs_link<LR, COMP>(k, fwd + (size_t)(kind * 4 + mu) * k.blk_bytes, p, mu, kind, cb, c, c[3], U);
#pragma unroll
          for (int q = 0; q < NG; ++q) {
            if (sub + q * ts < k.ngr) {
              cplx<SA> vs[G][3];
              GIO::load(k.in, (size_t)nb, k.ngr, sub + q * ts, vs);
#pragma unroll
              for (int s = 0; s < G; ++s) {
                const cplx<A> v[3] = {{A(vs[s][0].re), A(vs[s][0].im)},
                                      {A(vs[s][1].re), A(vs[s][1].im)},
                                      {A(vs[s][2].re), A(vs[s][2].im)}};
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                  for (int j = 0; j < 3; ++j) cmac(acc[q * G + s][i], U[3 * i + j], v[j]);
              }
            }
          }
        }
        // backward hop: - W_mu(x - hop mu)^dag in(x - hop mu)
        {
          const int nb = neighbour_cb(g, c, idx, mu, -hop);
          // a compressed long link sits at y = x - 3mu: only its t coordinate can change its fold sign
          const int yt = mu == 3 ? (c[3] >= hop ? c[3] - hop : c[3] - hop + g.L[3]) : c[3];
          cplx<A> U[9];
          mrhs_link<LR, COMP>(k, bwd + (size_t)(kind * 4 + mu) * k.blk_bytes, 1 - p, mu, kind, nb, c, yt, U);
#pragma unroll
          for (int q = 0; q < NG; ++q) {
            if (sub + q * ts < k.ngr) {
              cplx<SA> vs[G][3];
              GIO::load(k.in, (size_t)nb, k.ngr, sub + q * ts, vs);
#pragma unroll
              for (int s = 0; s < G; ++s) {
                const cplx<A> v[3] = {{A(vs[s][0].re), A(vs[s][0].im)},
                                      {A(vs[s][1].re), A(vs[s][1].im)},
                                      {A(vs[s][2].re), A(vs[s][2].im)}};
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                  for (int j = 0; j < 3; ++j) cmac_conj_sub(acc[q * G + s][i], U[3 * j + i], v[j]);
              }
            }
          }
        }
      }
    }

#pragma unroll
    for (int q = 0; q < NG; ++q) {
      if (sub + q * ts < k.ngr) {
        const int gq = sub + q * ts;
        cplx<SA> o[G][3];
        if (EPI == EPI_PLAIN) {
#pragma unroll
          for (int s = 0; s < G; ++s)
#pragma unroll
            for (int i = 0; i < 3; ++i) o[s][i] = {SA(acc[q * G + s][i].re), SA(acc[q * G + s][i].im)};
        } else {
          using EA = typename std::conditional<std::is_same<A, df64>::value, double, A>::type;
          cplx<SA> yv[G][3];
          GIO::load(k.y, (size_t)cb, k.ngr, gq, yv);
#pragma unroll
          for (int s = 0; s < G; ++s) {
            const EA a = EA(k.a[gq * G + s]);
            SA t = SA(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              o[s][i].re = SA(fma(a, EA(yv[s][i].re), -EA(acc[q * G + s][i].re)));
              o[s][i].im = SA(fma(a, EA(yv[s][i].im), -EA(acc[q * G + s][i].im)));
              t += yv[s][i].re * o[s][i].re + yv[s][i].im * o[s][i].im;
            }
            // the site's term in the arithmetic precision, summed over sites in FP64
            dot[q * G + s] += (double)t;
          }
        }
        GIO::store(k.out, (size_t)cb, k.ngr, gq, o);
      }
    }
  }

  if constexpr (EPI == EPI_AXPY) {
    if (k.partials == nullptr) return;  // uniform over the grid
    // lanes with the same sub hold the same vectors: sum over the sites of the warp first
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < NV; ++r)
      for (int off = ts; off < 32; off <<= 1) dot[r] += __shfl_xor_sync(0xffffffffu, dot[r], off);
    __shared__ double wred[8 * MRHS_MAX];  // [warp][sub * NV + r], blockDim <= 256
    const int N = k.ngr * G;
    if (lane < ts) {
#pragma unroll
      for (int r = 0; r < NV; ++r) {
        const int R = (lane + (r / G) * ts) * G + r % G;  // vector of granule lane + (r / G) ts
        if (R < N) wred[warp * MRHS_MAX + R] = dot[r];
      }
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    for (int R = threadIdx.x; R < N; R += blockDim.x) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += wred[w * MRHS_MAX + R];
      k.partials[(size_t)R * gridDim.x + blockIdx.x] = s;
    }
    if (last_block_done(k.counter)) {
      // one warp per vector: lanes stride over the blocks' partials, then a fixed shuffle tree
      for (int R = warp; R < N; R += nw) {
        const double s = warp_sum_partials(k.partials + (size_t)R * gridDim.x, gridDim.x);
        if (lane == 0) k.dot_out[R] = s;
      }
    }
  }
}

}  // namespace hisq
