// HISQ-type link smearing: fat links as weighted sums of parallel-transport paths (the link itself,
// the 3-, 5- and 7-link staples, the Lepage staple), long links as the Naik product of three links,
// and the projection onto U(3) between the two smearing levels of the HISQ action (the action of
// the paper's simulations, Sec. 1; the path coefficients are not in the paper and are inputs).
//
// One level, for each direction mu, runs three passes over the whole lattice (lexicographic sites)
// whose intermediates stay in HBM:
//   pass 1  S_{nu,s}(x): the staple of U_mu in direction s*nu, for the 3 transverse nu and s = +-,
//           and X_nu(x) = c5 U_mu(x) + c7 (S_{nu,+}(x) + S_{nu,-}(x))
//   pass 2  Y_a(x) = c3 U_mu(x) + sum_{b != a} sum_r staple_{b,r}[X_c](x),
//           c the transverse direction other than a and b
//   pass 3  F_mu(x) = c1 U_mu(x) + sum_a sum_r staple_{a,r}[Y_a + cL S_{a,r}](x)
//           L_mu(x) = cN U_mu(x) U_mu(x+mu) U_mu(x+2mu)
// where staple_{b,+}[X](x) = U_b(x) X(x+b) U_b(x+mu)^dag and staple_{b,-}[X](x) =
// U_b(x-b)^dag X(x-b) U_b(x-b+mu). Nesting the staples this way produces every 7-link path
// (a, b, c, mu, -c, -b, -a) once, every 5-link path (a, b, mu, -b, -a) once, the 3-link staples, and
// the Lepage path as the same-signed staple of a staple: 50 products of 3x3 complex matrices per
// site and direction (pass 1: 12, pass 2: 24, pass 3: 12, Naik: 2) instead of the ~400 of an explicit
// sum over the 84 paths.
//
// Arithmetic: FP64, or double-float (two FP32 words per real, ~2^-47 relative rounding) on the FP32
// pipe, which GB300 runs ~60x faster than its FP64 pipe. Inputs and outputs are binary64 either way.
#include <math.h>

#include <type_traits>

#include "internal.cuh"
#include "trace.h"
#include "tune.h"

namespace hisq {

bool is_device_ptr(const void* p);

namespace {

constexpr int SMEAR_BLOCK = 128;      // the conversion and projection kernels
constexpr int SMEAR_MAX_BLOCK = 256;  // the pass kernels: the tuner picks the block size up to this and one of
                                      // two register budgets (MINB 1: as many as the code wants; MINB 2:
                                      // 128 per thread, more resident warps, a few spills)

// One complex entry of an intermediate field: double2 for FP64 arithmetic, float4 (re.hi, re.lo,
// im.hi, im.lo) for double-float; 16 bytes either way. Fields are stored [entry 0..8][site].
template <typename T>
struct FieldIO;
template <>
struct FieldIO<double> {
  using S = double2;
  __device__ __forceinline__ static cplx<double> ld(const S* p) {
    const S v = __ldg(p);
    return {v.x, v.y};
  }
  // the entry, conjugated when c (a sign-bit flip on the integer pipe: the FP64 pipe is the bottleneck)
  __device__ __forceinline__ static cplx<double> ld_conj_if(const S* p, bool c) {
    const S v = __ldg(p);
    const long long m = c ? (long long)0x8000000000000000ull : 0ll;
    return {v.x, __longlong_as_double(__double_as_longlong(v.y) ^ m)};
  }
  __device__ __forceinline__ static cplx<double> ld_coherent(const S* p) {  // written by this kernel
    const S v = *p;
    return {v.x, v.y};
  }
  __device__ __forceinline__ static void st(S* p, const cplx<double>& c) { *p = make_double2(c.re, c.im); }
  __device__ __forceinline__ static cplx<double> from_f64(double2 v) { return {v.x, v.y}; }
  __device__ __forceinline__ static double2 to_f64(const cplx<double>& c) { return make_double2(c.re, c.im); }
  __device__ __forceinline__ static double coef(double c) { return c; }
  __device__ __forceinline__ static double zero() { return 0.0; }
};
template <>
struct FieldIO<df64> {
  using S = float4;
  __device__ __forceinline__ static cplx<df64> ld(const S* p) {
    const S v = __ldg(p);
    return {df64(v.x, v.y), df64(v.z, v.w)};
  }
  __device__ __forceinline__ static cplx<df64> ld_conj_if(const S* p, bool c) {
    const S v = __ldg(p);
    const unsigned m = c ? 0x80000000u : 0u;
    return {df64(v.x, v.y), df64(__uint_as_float(__float_as_uint(v.z) ^ m), __uint_as_float(__float_as_uint(v.w) ^ m))};
  }
  __device__ __forceinline__ static cplx<df64> ld_coherent(const S* p) {  // written by this kernel
    const S v = *p;
    return {df64(v.x, v.y), df64(v.z, v.w)};
  }
  __device__ __forceinline__ static void st(S* p, const cplx<df64>& c) {
    *p = make_float4(c.re.hi, c.re.lo, c.im.hi, c.im.lo);
  }
  __device__ __forceinline__ static cplx<df64> from_f64(double2 v) { return {df64(v.x), df64(v.y)}; }
  __device__ __forceinline__ static double2 to_f64(const cplx<df64>& c) {
    return make_double2((double)c.re, (double)c.im);
  }
  __device__ __forceinline__ static df64 coef(double c) { return df64(c); }
  __device__ __forceinline__ static df64 zero() { return df64(0.f, 0.f); }
};

template <typename T>
struct M3 {
  cplx<T> e[9];  // row-major
};

template <typename T>
__device__ __forceinline__ cplx<T> conj_c(const cplx<T>& a) {
  return {a.re, -a.im};
}

// m = f[s], or its conjugate transpose when dag
template <typename T>
__device__ __forceinline__ void load_m(M3<T>& m, const typename FieldIO<T>::S* f, size_t V, int s, bool dag) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      m.e[3 * i + j] = FieldIO<T>::ld_conj_if(f + (size_t)(dag ? 3 * j + i : 3 * i + j) * V + s, dag);
    }
}

template <typename T>
__device__ __forceinline__ void zero_m(M3<T>& m) {
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = {FieldIO<T>::zero(), FieldIO<T>::zero()};
}

template <typename T>
__device__ __forceinline__ void store_m(typename FieldIO<T>::S* f, size_t V, int s, const M3<T>& m) {
#pragma unroll
  for (int k = 0; k < 9; ++k) FieldIO<T>::st(f + (size_t)k * V + s, m.e[k]);
}

// m = a * f0[s] + b * (f1[s] + f2[s]); f2 may be null (m = a f0 + b f1), and f1 too (m = a f0)
template <typename T>
__device__ __forceinline__ void load_comb(M3<T>& m, const typename FieldIO<T>::S* f0, T a,
                                          const typename FieldIO<T>::S* f1, const typename FieldIO<T>::S* f2, T b,
                                          size_t V, int s) {
  const T z = FieldIO<T>::zero();
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const cplx<T> u = FieldIO<T>::ld(f0 + (size_t)k * V + s);
    cplx<T> r;
    r.re = fma(a, u.re, z);
    r.im = fma(a, u.im, z);
    if (f1) {
      cplx<T> w = FieldIO<T>::ld(f1 + (size_t)k * V + s);
      if (f2) {
        const cplx<T> w2 = FieldIO<T>::ld(f2 + (size_t)k * V + s);
        w.re = w.re + w2.re;
        w.im = w.im + w2.im;
      }
      r.re = fma(b, w.re, r.re);
      r.im = fma(b, w.im, r.im);
    }
    m.e[k] = r;
  }
}

// c = a b
template <typename T>
__device__ __forceinline__ void mul_nn(M3<T>& c, const M3<T>& a, const M3<T>& b) {
  const T z = FieldIO<T>::zero();
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<T> acc{z, z};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, a.e[3 * i + k], b.e[3 * k + j]);
      c.e[3 * i + j] = acc;
    }
}

// acc += a b
template <typename T>
__device__ __forceinline__ void mul_nn_acc(M3<T>& acc, const M3<T>& a, const M3<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc.e[3 * i + j], a.e[3 * i + k], b.e[3 * k + j]);
}

// Double-float 3x3 products with lazy renormalisation: each product of two double-float numbers is
// split exactly into the FP32 product of the high words and an error term (its FMA residual plus the
// two cross terms); the high parts of an output entry's terms are summed with error-free additions
// (Knuth's two-sum), all error terms in plain FP32, and the entry is renormalised once at the end
// instead of after every multiply-add. The real and imaginary parts run in the two lanes of the
// two-wide FP32 instructions.
__device__ __forceinline__ void df_dot_term(float2& S, float2& Lo, float2 ahi, float2 alo, float2 bhi, float2 blo) {
  const float2 p = __fmul2_rn(ahi, bhi);
  float2 e = __ffma2_rn(ahi, bhi, make_float2(-p.x, -p.y));
  e = __ffma2_rn(ahi, blo, e);
  e = __ffma2_rn(alo, bhi, e);
  const df64x2 t = df2_two_sum(S, p);
  S = t.hi;
  Lo = __fadd2_rn(Lo, __fadd2_rn(t.lo, e));
}

// (S, Lo) += x y for complex x, y: (re, im) lanes += (x.re, x.re)(y.re, y.im) + (-x.im, x.im)(y.im, y.re)
__device__ __forceinline__ void df_cmac_lazy(float2& S, float2& Lo, const cplx<df64>& x, const cplx<df64>& y) {
  df_dot_term(S, Lo, make_float2(x.re.hi, x.re.hi), make_float2(x.re.lo, x.re.lo), make_float2(y.re.hi, y.im.hi),
              make_float2(y.re.lo, y.im.lo));
  df_dot_term(S, Lo, make_float2(-x.im.hi, x.im.hi), make_float2(-x.im.lo, x.im.lo), make_float2(y.im.hi, y.re.hi),
              make_float2(y.im.lo, y.re.lo));
}

__device__ __forceinline__ void mul_nn_acc(M3<df64>& acc, const M3<df64>& a, const M3<df64>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<df64>& c = acc.e[3 * i + j];
      float2 S = make_float2(c.re.hi, c.im.hi), Lo = make_float2(c.re.lo, c.im.lo);
#pragma unroll
      for (int k = 0; k < 3; ++k) df_cmac_lazy(S, Lo, a.e[3 * i + k], b.e[3 * k + j]);
      const df64x2 r = df2_fast_two_sum(S, Lo);
      c = {df64(r.hi.x, r.lo.x), df64(r.hi.y, r.lo.y)};
    }
}

__device__ __forceinline__ void mul_nn(M3<df64>& c, const M3<df64>& a, const M3<df64>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float2 S = make_float2(0.f, 0.f), Lo = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < 3; ++k) df_cmac_lazy(S, Lo, a.e[3 * i + k], b.e[3 * k + j]);
      const df64x2 r = df2_fast_two_sum(S, Lo);
      c.e[3 * i + j] = {df64(r.hi.x, r.lo.x), df64(r.hi.y, r.lo.y)};
    }
}

template <typename T>
__device__ __forceinline__ void scale_m(M3<T>& m, T c) {
  const T z = FieldIO<T>::zero();
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    m.e[k].re = fma(c, m.e[k].re, z);
    m.e[k].im = fma(c, m.e[k].im, z);
  }
}

// Lexicographic coordinates of site s.
__device__ __forceinline__ void lex_coords(const Geom& g, int s, int c[4]) {
  c[0] = s % g.L[0];
  int r = s / g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
}

// Site s moved by k (|k| < L) along d; cd is s's coordinate along d.
__device__ __forceinline__ int step(const Geom& g, int s, int cd, int d, int k) {
  const int n = cd + k;
  int r = s + k * g.stride[d];
  if (n >= g.L[d]) r -= g.L[d] * g.stride[d];
  if (n < 0) r += g.L[d] * g.stride[d];
  return r;
}

// The j-th (0..2) direction other than mu, in increasing order.
__device__ __forceinline__ int transverse(int mu, int j) { return j + (j >= mu); }

// Links of the boundary layout [site][mu][9] complex128 into fields [mu][entry][site].
template <typename T>
__global__ void __launch_bounds__(SMEAR_BLOCK) k_to_fields(const double2* __restrict__ in,
                                                           typename FieldIO<T>::S* __restrict__ out, int V) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int e = blockIdx.y;  // mu * 9 + entry
  if (s >= V) return;
  FieldIO<T>::st(out + (size_t)e * V + s, FieldIO<T>::from_f64(__ldg(in + (size_t)s * 36 + e)));
}

// Each pass accumulates products A X C of three matrices: A and C are links U_b at the two ends of a
// staple (conjugate-transposed at load time for the backward half), X is the middle field. One loop
// iteration handles one (direction, sign), so each kernel holds a single copy of the two 3x3
// products: the double-float products are long instruction sequences, and one copy keeps the loop
// inside the instruction cache.

// Pass 1: the six one-signed staples of U_mu at every site, S_{nu,+} at field 2j, S_{nu,-} at 2j+1
// (nu = transverse(mu, j)), and the middle field of pass 2 for each transverse direction,
// X_j = c5 U_mu + c7 (S_{nu,+} + S_{nu,-}), at field j of Xf.
template <typename T, int MINB>
__global__ void __launch_bounds__(SMEAR_MAX_BLOCK, MINB) k_smear_staples(const typename FieldIO<T>::S* __restrict__ U,
                                                               typename FieldIO<T>::S* __restrict__ St,
                                                               typename FieldIO<T>::S* __restrict__ Xf, Geom g,
                                                               int mu, double c5, double c7) {
  using S = typename FieldIO<T>::S;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const size_t V = g.V;
  int c[4];
  lex_coords(g, s, c);
  const S* Umu = U + (size_t)mu * 9 * V;
#pragma unroll 1
  for (int it = 0; it < 6; ++it) {
    const int nu = transverse(mu, it >> 1);
    const bool bwd = it & 1;
    const S* Unu = U + (size_t)nu * 9 * V;
    // forward: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag; backward: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
    const int y0 = bwd ? step(g, s, c[nu], nu, -1) : s;
    M3<T> a, b, p, r;
    load_m(a, Unu, V, y0, bwd);
    load_m(b, Umu, V, bwd ? y0 : step(g, s, c[nu], nu, 1), false);
    mul_nn(p, a, b);
    load_m(a, Unu, V, step(g, y0, c[mu], mu, 1), !bwd);
    zero_m(r);
    mul_nn_acc(r, p, a);
    store_m(St + (size_t)it * 9 * V, V, s, r);
    if (bwd) {  // r = S_{nu,-}; S_{nu,+} was stored by this thread one iteration ago
      const S* Sp = St + (size_t)(it - 1) * 9 * V;
      S* Xj = Xf + (size_t)(it >> 1) * 9 * V;
      const T t5 = FieldIO<T>::coef(c5), t7 = FieldIO<T>::coef(c7), z = FieldIO<T>::zero();
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const cplx<T> u = FieldIO<T>::ld(Umu + (size_t)k * V + s);
        const cplx<T> sp = FieldIO<T>::ld_coherent(Sp + (size_t)k * V + s);
        cplx<T> x;
        x.re = fma(t7, sp.re + r.e[k].re, fma(t5, u.re, z));
        x.im = fma(t7, sp.im + r.e[k].im, fma(t5, u.im, z));
        FieldIO<T>::st(Xj + (size_t)k * V + s, x);
      }
    }
  }
}

// Pass 2: Y_a for the transverse direction a = transverse(mu, blockIdx.x % 3). The three values of a
// are neighbouring blocks, so the links and staples of a group of sites are read while in L2.
template <typename T, int MINB>
__global__ void __launch_bounds__(SMEAR_MAX_BLOCK, MINB) k_smear_middle(const typename FieldIO<T>::S* __restrict__ U,
                                                              const typename FieldIO<T>::S* __restrict__ Xf,
                                                              typename FieldIO<T>::S* __restrict__ Y, Geom g, int mu,
                                                              double c3) {
  using S = typename FieldIO<T>::S;
  const int ai = blockIdx.x % 3;
  const int s = (blockIdx.x / 3) * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const size_t V = g.V;
  int c[4];
  lex_coords(g, s, c);
  const S* Umu = U + (size_t)mu * 9 * V;
  M3<T> y;
  load_m(y, Umu, V, s, false);
  scale_m(y, FieldIO<T>::coef(c3));
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    const int bsel = it >> 1, bi = bsel + (bsel >= ai), ci = 3 - ai - bi;
    const bool bwd = it & 1;
    const int b = transverse(mu, bi);
    const S* Ub = U + (size_t)b * 9 * V;
    // forward: U_b(x) X(x+b) U_b(x+mu)^dag; backward: U_b(x-b)^dag X(x-b) U_b(x-b+mu);
    // X = c5 U_mu + c7 (S_{c,+} + S_{c,-}), formed by pass 1
    const int y0 = bwd ? step(g, s, c[b], b, -1) : s;
    M3<T> x, u, p;
    load_m(x, Xf + (size_t)ci * 9 * V, V, bwd ? y0 : step(g, s, c[b], b, 1), false);
    load_m(u, Ub, V, y0, bwd);
    mul_nn(p, u, x);
    load_m(u, Ub, V, step(g, y0, c[mu], mu, 1), !bwd);
    mul_nn_acc(y, p, u);
  }
  store_m(Y + (size_t)ai * 9 * V, V, s, y);
}

template <typename T>
__device__ __forceinline__ void store_link(double2* out, int s, int mu, const M3<T>& m) {
  double2* o = out + ((size_t)s * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) o[k] = FieldIO<T>::to_f64(m.e[k]);
}

// Pass 3: the fat link F_mu and (lng != null) the Naik link L_mu, written in the boundary layout. The
// Naik product is a seventh loop iteration, U_mu(x) [cN U_mu(x+mu)] U_mu(x+2mu), into a fresh
// accumulator.
template <typename T, int MINB>
__global__ void __launch_bounds__(SMEAR_MAX_BLOCK, MINB) k_smear_fat(const typename FieldIO<T>::S* __restrict__ U,
                                                           const typename FieldIO<T>::S* __restrict__ St,
                                                           const typename FieldIO<T>::S* __restrict__ Y,
                                                           double2* __restrict__ fat, double2* __restrict__ lng,
                                                           Geom g, int mu, double c1, double cL, double cN) {
  using S = typename FieldIO<T>::S;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const size_t V = g.V;
  int c[4];
  lex_coords(g, s, c);
  const S* Umu = U + (size_t)mu * 9 * V;
  const T one = FieldIO<T>::coef(1.0), tL = FieldIO<T>::coef(cL), tN = FieldIO<T>::coef(cN);
  const int s_mu = step(g, s, c[mu], mu, 1);
  M3<T> f;
  load_m(f, Umu, V, s, false);
  scale_m(f, FieldIO<T>::coef(c1));
  const int nit = lng ? 7 : 6;
#pragma unroll 1
  for (int it = 0; it < nit; ++it) {
    M3<T> z, u, p;
    const S* Ua;
    int y0, sc;
    bool bwd;
    if (it < 6) {
      // forward: U_a(x) Z(x+a) U_a(x+mu)^dag; backward: U_a(x-a)^dag Z(x-a) U_a(x-a+mu);
      // Z = Y_a + cL S_{a,sign}
      const int ai = it >> 1, a = transverse(mu, ai);
      bwd = it & 1;
      Ua = U + (size_t)a * 9 * V;
      y0 = bwd ? step(g, s, c[a], a, -1) : s;
      sc = step(g, y0, c[mu], mu, 1);
      load_comb(z, Y + (size_t)ai * 9 * V, one, cL != 0.0 ? St + (size_t)it * 9 * V : (const S*)nullptr,
                (const S*)nullptr, tL, V, bwd ? y0 : step(g, s, c[a], a, 1));
    } else {
      store_link(fat, s, mu, f);
      zero_m(f);
      bwd = false;
      Ua = Umu;
      y0 = s;
      sc = step(g, s_mu, c[mu] + 1 < g.L[mu] ? c[mu] + 1 : 0, mu, 1);
      load_comb(z, Umu, tN, (const S*)nullptr, (const S*)nullptr, tN, V, s_mu);
    }
    load_m(u, Ua, V, y0, bwd);
    mul_nn(p, u, z);
    load_m(u, Ua, V, sc, !bwd && it < 6);
    mul_nn_acc(f, p, u);
  }
  store_link(lng ? lng : fat, s, mu, f);
}

// W -> W (W^dag W)^{-1/2} for every link (matrix products in T, eigenvalues in FP64). The inverse square root of the Hermitian
// Q = W^dag W is the polynomial f0 + f1 Q + f2 Q^2 that takes the value g^{-1/2} at each eigenvalue g
// of Q (Cayley-Hamilton); with s_i = sqrt(g_i), u = s1 + s2 + s3, v = s1 s2 + s1 s3 + s2 s3, w = s1 s2 s3:
//   f0 = (u v^2 - w (u^2 + v)) / d,  f1 = (2 u v - u^3 - w) / d,  f2 = u / d,  d = w (u v - w).
// The eigenvalues come from the trigonometric solution of the characteristic cubic of Q - (tr Q / 3).
// A link whose Q is not positive definite (or not finite) sets bit 4 of *flag and is copied unchanged.
template <typename T>
__global__ void __launch_bounds__(SMEAR_BLOCK) k_project_u3(double2* out, const double2* in, long long nlinks,
                                                            int* flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlinks) return;
  const T z = FieldIO<T>::zero();
  cplx<T> W[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) W[k] = FieldIO<T>::from_f64(in[i * 9 + k]);
  cplx<T> Q[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<T> acc{z, z};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, conj_c(W[3 * k + a]), W[3 * k + b]);
      Q[3 * a + b] = acc;
    }
  // the eigenvalues (a few scalars) in FP64 whatever the arithmetic of the matrix products
  const double c0 = ((double)Q[0].re + (double)Q[4].re + (double)Q[8].re) / 3.0;
  const double d0 = (double)Q[0].re - c0, d1 = (double)Q[4].re - c0, d2 = (double)Q[8].re - c0;
  const cplx<double> q01{(double)Q[1].re, (double)Q[1].im}, q02{(double)Q[2].re, (double)Q[2].im},
      q12{(double)Q[5].re, (double)Q[5].im};
  const double n01 = q01.re * q01.re + q01.im * q01.im, n02 = q02.re * q02.re + q02.im * q02.im,
               n12 = q12.re * q12.re + q12.im * q12.im;
  const double p = (d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * (n01 + n02 + n12)) / 6.0;
  // det(Q - c0) of a Hermitian matrix; Re(q01 q12 conj(q02)) is the product of the three off-diagonals
  const double re3 = (q01.re * q12.re - q01.im * q12.im) * q02.re + (q01.re * q12.im + q01.im * q12.re) * q02.im;
  const double det = d0 * d1 * d2 + 2.0 * re3 - d0 * n12 - d1 * n02 - d2 * n01;
  double g[3] = {c0, c0, c0};
  if (p > 0.0) {
    const double sp = sqrt(p);
    double r = 0.5 * det / (p * sp);
    r = fmin(1.0, fmax(-1.0, r));
    const double phi = acos(r) / 3.0;
    const double two_pi_3 = 2.0943951023931957;
    g[0] = c0 + 2.0 * sp * cos(phi);
    g[1] = c0 + 2.0 * sp * cos(phi + two_pi_3);
    g[2] = c0 + 2.0 * sp * cos(phi - two_pi_3);
  }
  if (!(g[0] > 0.0 && g[1] > 0.0 && g[2] > 0.0 && isfinite(g[0] + g[1] + g[2]))) {
    atomicOr(flag, 4);
#pragma unroll
    for (int k = 0; k < 9; ++k) out[i * 9 + k] = in[i * 9 + k];
    return;
  }
  const double s0 = sqrt(g[0]), s1 = sqrt(g[1]), s2 = sqrt(g[2]);
  const double u = s0 + s1 + s2, v = s0 * s1 + s0 * s2 + s1 * s2, w = s0 * s1 * s2;
  const double inv_d = 1.0 / (w * (u * v - w));
  const T f0 = FieldIO<T>::coef((u * v * v - w * (u * u + v)) * inv_d),
          f1 = FieldIO<T>::coef((2.0 * u * v - u * u * u - w) * inv_d), f2 = FieldIO<T>::coef(u * inv_d);
  // X = f0 + f1 Q + f2 Q^2
  cplx<T> X[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<T> q2{z, z};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(q2, Q[3 * a + k], Q[3 * k + b]);
      X[3 * a + b] = {fma(f1, Q[3 * a + b].re, fma(f2, q2.re, a == b ? f0 : z)), fma(f1, Q[3 * a + b].im, fma(f2, q2.im, z))};
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<T> acc{z, z};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, W[3 * a + k], X[3 * k + b]);
      out[i * 9 + 3 * a + b] = FieldIO<T>::to_f64(acc);
    }
}

// One pass kernel with its launch shape chosen by the tuner: a register budget (MINB 1 or 2) and the
// block size. All three passes are idempotent (their outputs are not read), so they can be timed.
template <typename Kern, typename Launch>
int launch_pass(hisq_ctx* ctx, const char* key, Kern k1, Kern k2, Launch launch) {
  TuneVariant v[2] = {{(const void*)k1, [&](int b) { return launch(k1, b); }},
                      {(const void*)k2, [&](int b) { return launch(k2, b); }}};
  int vi = 0, block = SMEAR_BLOCK;
  int rc = tuned_variant(ctx, key, v, 2, &vi, &block);
  if (rc) return rc;
  HISQ_CUDA(v[vi].run(block));
  note_launch(ctx);
  return HISQ_OK;
}

inline unsigned blocks_for(size_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T>
int smear_level(hisq_ctx* ctx, double* fat, double* lng, const double* thin, const hisq_smear_coeffs& cf) {
  using S = typename FieldIO<T>::S;
  const Geom g = ctx->g;
  const size_t V = g.V;
  cudaStream_t st = ctx->stream;
  S* U = (S*)workspace(ctx, "smear_thin", 36 * V * sizeof(S));
  S* Sf = (S*)workspace(ctx, "smear_staples", 54 * V * sizeof(S));
  S* Y = (S*)workspace(ctx, "smear_middle", 27 * V * sizeof(S));
  S* Xf = (S*)workspace(ctx, "smear_x", 27 * V * sizeof(S));
  if (!U || !Sf || !Y || !Xf) return set_error(HISQ_ENOMEM, "smearing workspaces (%zu bytes)", 144 * V * sizeof(S));
  k_to_fields<T><<<dim3(blocks_for(V, SMEAR_BLOCK), 36), SMEAR_BLOCK, 0, st>>>((const double2*)thin, U, g.V);
  HISQ_CUDA(cudaGetLastError());
  note_launch(ctx);
  const bool dd = std::is_same<T, df64>::value;
  const double c3 = cf.three_staple, c5 = cf.five_staple, c7 = cf.seven_staple, c1 = cf.one_link, cL = cf.lepage,
               cN = cf.naik;
  double2 *f2 = (double2*)fat, *l2 = (double2*)lng;
  for (int mu = 0; mu < 4; ++mu) {
    int rc = launch_pass(ctx, dd ? "smear/staples/df64" : "smear/staples/f64", k_smear_staples<T, 1>,
                         k_smear_staples<T, 2>, [&](decltype(&k_smear_staples<T, 1>) k, int b) {
                           k<<<blocks_for(V, b), b, 0, st>>>(U, Sf, Xf, g, mu, c5, c7);
                           return cudaGetLastError();
                         });
    if (rc) return rc;
    rc = launch_pass(ctx, dd ? "smear/middle/df64" : "smear/middle/f64", k_smear_middle<T, 1>, k_smear_middle<T, 2>,
                     [&](decltype(&k_smear_middle<T, 1>) k, int b) {
                       k<<<3 * blocks_for(V, b), b, 0, st>>>(U, Xf, Y, g, mu, c3);
                       return cudaGetLastError();
                     });
    if (rc) return rc;
    rc = launch_pass(ctx, dd ? "smear/fat/df64" : "smear/fat/f64", k_smear_fat<T, 1>, k_smear_fat<T, 2>,
                     [&](decltype(&k_smear_fat<T, 1>) k, int b) {
                       k<<<blocks_for(V, b), b, 0, st>>>(U, Sf, Y, f2, l2, g, mu, c1, cL, cN);
                       return cudaGetLastError();
                     });
    if (rc) return rc;
  }
  return HISQ_OK;
}

// The projection with its matrix products in FP64 or (prec HISQ_DF64) double-float.
int launch_project(hisq_ctx* ctx, double* out, const double* in, int prec) {
  const long long n = (long long)ctx->g.V * 4;
  const unsigned nb = (unsigned)((n + SMEAR_BLOCK - 1) / SMEAR_BLOCK);
  if (prec == HISQ_DF64)
    k_project_u3<df64><<<nb, SMEAR_BLOCK, 0, ctx->stream>>>((double2*)out, (const double2*)in, n, ctx->d_flag);
  else
    k_project_u3<double><<<nb, SMEAR_BLOCK, 0, ctx->stream>>>((double2*)out, (const double2*)in, n, ctx->d_flag);
  note_launch(ctx);
  HISQ_CUDA(cudaGetLastError());
  return HISQ_OK;
}

int read_project_flag(hisq_ctx* ctx) {
  int flag = 0;
  HISQ_CUDA(cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
  if (flag & 4) return set_error(HISQ_EINVAL, "U(3) projection: a link W with W^dag W not positive definite");
  return HISQ_OK;
}

bool overlap(const void* a, const void* b, size_t bytes) {
  const char *pa = (const char*)a, *pb = (const char*)b;
  return a && b && pa < pb + bytes && pb < pa + bytes;
}

int check_field(const hisq_ctx* ctx, const void* p, const char* what) {
  if (!is_device_ptr(p)) return set_error(HISQ_EINVAL, "%s: not a device pointer", what);
  if ((uintptr_t)p % 16) return set_error(HISQ_EINVAL, "%s: not 16-byte aligned", what);
  (void)ctx;
  return HISQ_OK;
}

int check_smear_args(hisq_ctx* c, const double* fat, const double* lng, const double* thin,
                     const hisq_smear_coeffs* cf, int prec) {
  if (!c || !fat || !thin || !cf) return set_error(HISQ_EINVAL, "null argument");
  if (prec != HISQ_F64 && prec != HISQ_DF64)
    return set_error(HISQ_EINVAL, "smearing arithmetic %d: HISQ_F64 or HISQ_DF64 only", prec);
  const double v[6] = {cf->one_link, cf->three_staple, cf->five_staple, cf->seven_staple, cf->lepage, cf->naik};
  for (double x : v)
    if (!isfinite(x)) return set_error(HISQ_EINVAL, "non-finite path coefficient");
  int rc;
  if ((rc = check_field(c, thin, "thin links")) || (rc = check_field(c, fat, "fat links"))) return rc;
  if (lng && (rc = check_field(c, lng, "long links"))) return rc;
  const size_t bytes = (size_t)c->g.V * 4 * 18 * sizeof(double);
  if (overlap(fat, thin, bytes) || overlap(lng, thin, bytes) || overlap(fat, lng, bytes))
    return set_error(HISQ_EINVAL, "output links overlap the input links or each other");
  return HISQ_OK;
}

int smear_dispatch(hisq_ctx* c, double* fat, double* lng, const double* thin, const hisq_smear_coeffs& cf, int prec) {
  return prec == HISQ_DF64 ? smear_level<df64>(c, fat, lng, thin, cf) : smear_level<double>(c, fat, lng, thin, cf);
}

}  // namespace
}  // namespace hisq

using namespace hisq;

extern "C" int hisq_smear(hisq_ctx* c, double* fat, double* lng, const double* thin, const hisq_smear_coeffs* cf,
                          int prec) {
  TraceRange trace("hisq_smear");
  int rc = check_smear_args(c, fat, lng, thin, cf, prec);
  if (rc) return rc;
  return smear_dispatch(c, fat, lng, thin, *cf, prec);
}

extern "C" int hisq_project_u3(hisq_ctx* c, double* out, const double* in) {
  TraceRange trace("hisq_project_u3");
  if (!c || !out || !in) return set_error(HISQ_EINVAL, "null argument");
  int rc;
  if ((rc = check_field(c, in, "input links")) || (rc = check_field(c, out, "output links"))) return rc;
  const size_t bytes = (size_t)c->g.V * 4 * 18 * sizeof(double);
  if (out != in && overlap(out, in, bytes)) return set_error(HISQ_EINVAL, "output links partly overlap the input");
  HISQ_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  if ((rc = launch_project(c, out, in, HISQ_F64))) return rc;
  return read_project_flag(c);
}

extern "C" int hisq_hisq_links(hisq_ctx* c, double* fat, double* lng, const double* thin,
                               const hisq_smear_coeffs* level1, const hisq_smear_coeffs* level2, int prec) {
  TraceRange trace("hisq_hisq_links");
  int rc = check_smear_args(c, fat, lng, thin, level2, prec);
  if (rc) return rc;
  if (!level1) return set_error(HISQ_EINVAL, "null argument");
  rc = check_smear_args(c, fat, nullptr, thin, level1, prec);
  if (rc) return rc;
  double* w = (double*)workspace(c, "smear_level1", (size_t)c->g.V * 4 * 18 * sizeof(double));
  if (!w) return set_error(HISQ_ENOMEM, "level-1 links");
  HISQ_CUDA(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  if ((rc = smear_dispatch(c, w, nullptr, thin, *level1, prec))) return rc;
  if ((rc = launch_project(c, w, w, prec))) return rc;
  if ((rc = smear_dispatch(c, fat, lng, w, *level2, prec))) return rc;
  return read_project_flag(c);
}
