// HISQ-type link smearing: fat links as weighted sums of parallel-transport paths (the link itself,
// the 3-, 5- and 7-link staples, the Lepage staple), long links as the Naik product of three links,
// and the projection onto U(3) between the two smearing levels of the HISQ action (the action of
// the paper's simulations, Sec. 1; the path coefficients are not in the paper and are inputs).
//
// One level, for each direction mu, runs three passes over the whole lattice (lexicographic sites)
// whose intermediates stay in HBM:
//   pass 1  S_{nu,s}(x): the staple of U_mu in direction s*nu, for the 3 transverse nu and s = +-
//   pass 2  Y_a(x) = c3 U_mu(x) + sum_{b != a} sum_r staple_{b,r}[c5 U_mu + c7 (S_{c,+} + S_{c,-})](x),
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

#include "internal.cuh"
#include "trace.h"

namespace hisq {

bool is_device_ptr(const void* p);

namespace {

constexpr int SMEAR_BLOCK = 128;

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

template <typename T>
__device__ __forceinline__ void load_m(M3<T>& m, const typename FieldIO<T>::S* f, size_t V, int s) {
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = FieldIO<T>::ld(f + (size_t)k * V + s);
}

template <typename T>
__device__ __forceinline__ void store_m(typename FieldIO<T>::S* f, size_t V, int s, const M3<T>& m) {
#pragma unroll
  for (int k = 0; k < 9; ++k) FieldIO<T>::st(f + (size_t)k * V + s, m.e[k]);
}

// m = a * f0[s] + b * (f1[s] + f2[s]) (f2 may be null: m = a f0 + b f1)
template <typename T>
__device__ __forceinline__ void load_comb(M3<T>& m, const typename FieldIO<T>::S* f0, T a,
                                          const typename FieldIO<T>::S* f1, const typename FieldIO<T>::S* f2, T b,
                                          size_t V, int s) {
  const T z = FieldIO<T>::zero();
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const cplx<T> u = FieldIO<T>::ld(f0 + (size_t)k * V + s);
    cplx<T> w = FieldIO<T>::ld(f1 + (size_t)k * V + s);
    if (f2) {
      const cplx<T> w2 = FieldIO<T>::ld(f2 + (size_t)k * V + s);
      w.re = w.re + w2.re;
      w.im = w.im + w2.im;
    }
    cplx<T> r;
    r.re = fma(a, u.re, z);
    r.im = fma(a, u.im, z);
    r.re = fma(b, w.re, r.re);
    r.im = fma(b, w.im, r.im);
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

// c = a^dag b
template <typename T>
__device__ __forceinline__ void mul_dn(M3<T>& c, const M3<T>& a, const M3<T>& b) {
  const T z = FieldIO<T>::zero();
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<T> acc{z, z};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, conj_c(a.e[3 * k + i]), b.e[3 * k + j]);
      c.e[3 * i + j] = acc;
    }
}

// c = a b^dag
template <typename T>
__device__ __forceinline__ void mul_nd(M3<T>& c, const M3<T>& a, const M3<T>& b) {
  const T z = FieldIO<T>::zero();
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cplx<T> acc{z, z};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, a.e[3 * i + k], conj_c(b.e[3 * j + k]));
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

// acc += a b^dag
template <typename T>
__device__ __forceinline__ void mul_nd_acc(M3<T>& acc, const M3<T>& a, const M3<T>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc.e[3 * i + j], a.e[3 * i + k], conj_c(b.e[3 * j + k]));
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

// Pass 1: the six one-signed staples of U_mu at every site.
template <typename T>
__global__ void __launch_bounds__(SMEAR_BLOCK) k_smear_staples(const typename FieldIO<T>::S* __restrict__ U,
                                                               typename FieldIO<T>::S* __restrict__ St, Geom g,
                                                               int mu) {
  using S = typename FieldIO<T>::S;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const size_t V = g.V;
  int c[4];
  lex_coords(g, s, c);
  const S* Umu = U + (size_t)mu * 9 * V;
  const int s_mu = step(g, s, c[mu], mu, 1);
#pragma unroll 1
  for (int j = 0; j < 3; ++j) {
    const int nu = transverse(mu, j);
    const S* Unu = U + (size_t)nu * 9 * V;
    M3<T> a, b, p, r;
    // U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
    load_m(a, Unu, V, s);
    load_m(b, Umu, V, step(g, s, c[nu], nu, 1));
    mul_nn(p, a, b);
    load_m(a, Unu, V, s_mu);
    mul_nd(r, p, a);
    store_m(St + (size_t)(2 * j) * 9 * V, V, s, r);
    // U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
    const int m = step(g, s, c[nu], nu, -1);
    load_m(a, Unu, V, m);
    load_m(b, Umu, V, m);
    mul_dn(p, a, b);
    load_m(a, Unu, V, step(g, m, c[mu], mu, 1));
    mul_nn(r, p, a);
    store_m(St + (size_t)(2 * j + 1) * 9 * V, V, s, r);
  }
}

// Pass 2: Y_a for the transverse direction a = transverse(mu, blockIdx.y).
template <typename T>
__global__ void __launch_bounds__(SMEAR_BLOCK) k_smear_middle(const typename FieldIO<T>::S* __restrict__ U,
                                                              const typename FieldIO<T>::S* __restrict__ St,
                                                              typename FieldIO<T>::S* __restrict__ Y, Geom g, int mu,
                                                              double c3, double c5, double c7) {
  using S = typename FieldIO<T>::S;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const size_t V = g.V;
  const int ai = blockIdx.y;
  int c[4];
  lex_coords(g, s, c);
  const S* Umu = U + (size_t)mu * 9 * V;
  const T t5 = FieldIO<T>::coef(c5), t7 = FieldIO<T>::coef(c7);
  M3<T> y;
  load_m(y, Umu, V, s);
  scale_m(y, FieldIO<T>::coef(c3));
#pragma unroll 1
  for (int bi = 0; bi < 3; ++bi) {
    if (bi == ai) continue;
    const int b = transverse(mu, bi), ci = 3 - ai - bi;
    const S* Ub = U + (size_t)b * 9 * V;
    const S* Sp = St + (size_t)(2 * ci) * 9 * V;
    const S* Sm = St + (size_t)(2 * ci + 1) * 9 * V;
    M3<T> x, u, p;
    // U_b(x) X(x+b) U_b(x+mu)^dag, X = c5 U_mu + c7 (S_{c,+} + S_{c,-})
    load_comb(x, Umu, t5, Sp, Sm, t7, V, step(g, s, c[b], b, 1));
    load_m(u, Ub, V, s);
    mul_nn(p, u, x);
    load_m(u, Ub, V, step(g, s, c[mu], mu, 1));
    mul_nd_acc(y, p, u);
    // U_b(x-b)^dag X(x-b) U_b(x-b+mu)
    const int m = step(g, s, c[b], b, -1);
    load_comb(x, Umu, t5, Sp, Sm, t7, V, m);
    load_m(u, Ub, V, m);
    mul_dn(p, u, x);
    load_m(u, Ub, V, step(g, m, c[mu], mu, 1));
    mul_nn_acc(y, p, u);
  }
  store_m(Y + (size_t)ai * 9 * V, V, s, y);
}

// Pass 3: the fat link F_mu and (lng != null) the Naik link L_mu, written in the boundary layout.
template <typename T>
__global__ void __launch_bounds__(SMEAR_BLOCK) k_smear_fat(const typename FieldIO<T>::S* __restrict__ U,
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
  const T one = FieldIO<T>::coef(1.0), tL = FieldIO<T>::coef(cL);
  const int s_mu = step(g, s, c[mu], mu, 1);
  M3<T> f;
  load_m(f, Umu, V, s);
  scale_m(f, FieldIO<T>::coef(c1));
#pragma unroll 1
  for (int ai = 0; ai < 3; ++ai) {
    const int a = transverse(mu, ai);
    const S* Ua = U + (size_t)a * 9 * V;
    const S* Ya = Y + (size_t)ai * 9 * V;
    M3<T> z, u, p;
    // U_a(x) Z(x+a) U_a(x+mu)^dag, Z = Y_a + cL S_{a,+}
    const int sp = step(g, s, c[a], a, 1);
    if (cL != 0.0)
      load_comb(z, Ya, one, St + (size_t)(2 * ai) * 9 * V, (const S*)nullptr, tL, V, sp);
    else
      load_m(z, Ya, V, sp);
    load_m(u, Ua, V, s);
    mul_nn(p, u, z);
    load_m(u, Ua, V, s_mu);
    mul_nd_acc(f, p, u);
    // U_a(x-a)^dag Z(x-a) U_a(x-a+mu), Z = Y_a + cL S_{a,-}
    const int m = step(g, s, c[a], a, -1);
    if (cL != 0.0)
      load_comb(z, Ya, one, St + (size_t)(2 * ai + 1) * 9 * V, (const S*)nullptr, tL, V, m);
    else
      load_m(z, Ya, V, m);
    load_m(u, Ua, V, m);
    mul_dn(p, u, z);
    load_m(u, Ua, V, step(g, m, c[mu], mu, 1));
    mul_nn_acc(f, p, u);
  }
  double2* out = fat + ((size_t)s * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) out[k] = FieldIO<T>::to_f64(f.e[k]);
  if (lng) {
    M3<T> a, b, p;
    load_m(a, Umu, V, s);
    load_m(b, Umu, V, s_mu);
    mul_nn(p, a, b);
    load_m(a, Umu, V, step(g, s_mu, (c[mu] + 1) % g.L[mu], mu, 1));
    mul_nn(f, p, a);
    scale_m(f, FieldIO<T>::coef(cN));
    double2* lo = lng + ((size_t)s * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) lo[k] = FieldIO<T>::to_f64(f.e[k]);
  }
}

// W -> W (W^dag W)^{-1/2} for every link, in FP64. The inverse square root of the Hermitian
// Q = W^dag W is the polynomial f0 + f1 Q + f2 Q^2 that takes the value g^{-1/2} at each eigenvalue g
// of Q (Cayley-Hamilton); with s_i = sqrt(g_i), u = s1 + s2 + s3, v = s1 s2 + s1 s3 + s2 s3, w = s1 s2 s3:
//   f0 = (u v^2 - w (u^2 + v)) / d,  f1 = (2 u v - u^3 - w) / d,  f2 = u / d,  d = w (u v - w).
// The eigenvalues come from the trigonometric solution of the characteristic cubic of Q - (tr Q / 3).
// A link whose Q is not positive definite (or not finite) sets bit 4 of *flag and is copied unchanged.
__global__ void __launch_bounds__(SMEAR_BLOCK) k_project_u3(double2* out, const double2* in, long long nlinks,
                                                            int* flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlinks) return;
  cplx<double> W[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 v = in[i * 9 + k];
    W[k] = {v.x, v.y};
  }
  cplx<double> Q[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<double> acc{0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, conj_c(W[3 * k + a]), W[3 * k + b]);
      Q[3 * a + b] = acc;
    }
  const double c0 = (Q[0].re + Q[4].re + Q[8].re) / 3.0;
  const double d0 = Q[0].re - c0, d1 = Q[4].re - c0, d2 = Q[8].re - c0;
  const cplx<double> q01 = Q[1], q02 = Q[2], q12 = Q[5];
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
    for (int k = 0; k < 9; ++k) out[i * 9 + k] = make_double2(W[k].re, W[k].im);
    return;
  }
  const double s0 = sqrt(g[0]), s1 = sqrt(g[1]), s2 = sqrt(g[2]);
  const double u = s0 + s1 + s2, v = s0 * s1 + s0 * s2 + s1 * s2, w = s0 * s1 * s2;
  const double inv_d = 1.0 / (w * (u * v - w));
  const double f0 = (u * v * v - w * (u * u + v)) * inv_d, f1 = (2.0 * u * v - u * u * u - w) * inv_d, f2 = u * inv_d;
  // X = f0 + f1 Q + f2 Q^2
  cplx<double> X[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<double> q2{0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(q2, Q[3 * a + k], Q[3 * k + b]);
      X[3 * a + b] = {f1 * Q[3 * a + b].re + f2 * q2.re + (a == b ? f0 : 0.0), f1 * Q[3 * a + b].im + f2 * q2.im};
    }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      cplx<double> acc{0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, W[3 * a + k], X[3 * k + b]);
      out[i * 9 + 3 * a + b] = make_double2(acc.re, acc.im);
    }
}

template <typename T>
int smear_level(hisq_ctx* ctx, double* fat, double* lng, const double* thin, const hisq_smear_coeffs& cf) {
  using S = typename FieldIO<T>::S;
  const Geom& g = ctx->g;
  const size_t V = g.V;
  S* U = (S*)workspace(ctx, "smear_thin", 36 * V * sizeof(S));
  S* St = (S*)workspace(ctx, "smear_staples", 54 * V * sizeof(S));
  S* Y = (S*)workspace(ctx, "smear_middle", 27 * V * sizeof(S));
  if (!U || !St || !Y) return set_error(HISQ_ENOMEM, "smearing workspaces (%zu bytes)", 117 * V * sizeof(S));
  const unsigned nb = (unsigned)((V + SMEAR_BLOCK - 1) / SMEAR_BLOCK);
  k_to_fields<T><<<dim3(nb, 36), SMEAR_BLOCK, 0, ctx->stream>>>((const double2*)thin, U, g.V);
  for (int mu = 0; mu < 4; ++mu) {
    k_smear_staples<T><<<nb, SMEAR_BLOCK, 0, ctx->stream>>>(U, St, g, mu);
    k_smear_middle<T><<<dim3(nb, 3), SMEAR_BLOCK, 0, ctx->stream>>>(U, St, Y, g, mu, cf.three_staple,
                                                                    cf.five_staple, cf.seven_staple);
    k_smear_fat<T><<<nb, SMEAR_BLOCK, 0, ctx->stream>>>(U, St, Y, (double2*)fat, (double2*)lng, g, mu,
                                                        cf.one_link, cf.lepage, cf.naik);
  }
  note_launch(ctx, 13);
  HISQ_CUDA(cudaGetLastError());
  return HISQ_OK;
}

int launch_project(hisq_ctx* ctx, double* out, const double* in) {
  const long long n = (long long)ctx->g.V * 4;
  k_project_u3<<<(unsigned)((n + SMEAR_BLOCK - 1) / SMEAR_BLOCK), SMEAR_BLOCK, 0, ctx->stream>>>(
      (double2*)out, (const double2*)in, n, ctx->d_flag);
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
  if ((rc = launch_project(c, out, in))) return rc;
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
  if ((rc = launch_project(c, w, w))) return rc;
  if ((rc = smear_dispatch(c, fat, lng, w, *level2, prec))) return rc;
  return read_project_flag(c);
}
