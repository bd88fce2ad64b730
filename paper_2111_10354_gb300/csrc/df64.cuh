// Double-float ("df64") arithmetic: a real number held as an unevaluated sum hi + lo of two FP32
// values, carried out on the FP32 pipe. GB300 runs ~2 FP64 operations per clock per SM against
// 128 FP32 FMAs, so the FP64 Dslash is bound by its FP64 arithmetic at ~0.37 of HBM; the same
// operator in double-float arithmetic has 2^-47 relative rounding per operation (48-bit
// significand instead of 53) and is bound by HBM again.
//
// Algorithms: the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2):
// two_sum(a, b) = (s, e) with s = fl(a + b) and s + e = a + b exactly; the product error
// fma(a, b, -fl(a*b)) is exact. Every operation is written with the round-to-nearest
// intrinsics so the compiler neither contracts nor reorders them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hisq {

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // From a double with integer operations only (no FP64 instruction): hi keeps the first 24
  // significant bits of d, lo the remaining 29 rounded to 24, so |d - hi - lo| <= 2^-47 |d|.
  // |d| < 2^-100 (and zero) becomes 0; |d| must be below 2^127.
  __device__ __forceinline__ explicit df64(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const int e = (int)((hw >> 20) & 0x7ffu);
    const unsigned sign = hw & 0x80000000u;
    if (e < 1023 - 100) {
      hi = 0.f;
      lo = 0.f;
      return;
    }
    hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    // remaining bits: m29 * 2^(e - 1075) = (m29 * 2^-29) * 2^(e - 1046), both factors exact floats
    const float m = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), 1.862645149230957e-09f /* 2^-29 */);
    const float l = __fmul_rn(m, __uint_as_float((unsigned)(e - 919) << 23));
    lo = __uint_as_float(__float_as_uint(l) | sign);
  }
  // To a double: each part converted exactly by integer operations, then one FP64 add.
  __device__ __forceinline__ explicit operator double() const { return widen(hi) + widen(lo); }
  __device__ __forceinline__ static double widen(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned ef = (b >> 23) & 0xffu;
    if (ef == 0u) return 0.0;  // zero (FP32 subnormals do not arise from the splits above)
    const unsigned long long bits = ((unsigned long long)(b & 0x80000000u) << 32) |
                                    ((unsigned long long)(ef + 896u) << 52) |
                                    ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
  }
  __device__ __forceinline__ df64 operator-() const { return df64(-hi, -lo); }
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
  return df64(s, e);
}

// s + e = a + b exactly when |a| >= |b| (Dekker); used to renormalise.
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

using ::fma;  // the FP32/FP64 overloads stay visible next to the double-float one

// a * b + c in double-float: the exact product of the high parts, the cross terms in FP32,
// an error-free sum with c's high part, then one renormalisation.
__device__ __forceinline__ df64 fma(const df64& a, const df64& b, const df64& c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  const df64 s = df_two_sum(c.hi, p);
  const float t = __fadd_rn(s.lo, __fadd_rn(c.lo, pe));
  return df_fast_two_sum(s.hi, t);
}

__device__ __forceinline__ df64 operator+(const df64& a, const df64& b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// Two double-float numbers side by side (lane x, lane y), for Blackwell's two-wide FP32 instructions
// (one FFMA2/FADD2/FMUL2 does the same operation on both lanes): a complex multiply-accumulate
// updates the real and imaginary parts of its accumulator in the two lanes at once.
struct df64x2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 df2_sub(float2 a, float2 b) {  // a - b, one rounding (b * -1 is exact)
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

__device__ __forceinline__ df64x2 df2_two_sum(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  const float2 bv = df2_sub(s, a);
  return {s, __fadd2_rn(df2_sub(a, df2_sub(s, bv)), df2_sub(b, bv))};
}

__device__ __forceinline__ df64x2 df2_fast_two_sum(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  return {s, df2_sub(b, df2_sub(s, a))};
}

// Lane-wise a * b + c, the same steps as the scalar fma above.
__device__ __forceinline__ df64x2 df2_fma(const df64x2& a, const df64x2& b, const df64x2& c) {
  const float2 p = __fmul2_rn(a.hi, b.hi);
  float2 pe = __ffma2_rn(a.hi, b.hi, make_float2(-p.x, -p.y));
  pe = __ffma2_rn(a.hi, b.lo, pe);
  pe = __ffma2_rn(a.lo, b.hi, pe);
  const df64x2 s = df2_two_sum(c.hi, p);
  const float2 t = __fadd2_rn(s.lo, __fadd2_rn(c.lo, pe));
  return df2_fast_two_sum(s.hi, t);
}

}  // namespace hisq
