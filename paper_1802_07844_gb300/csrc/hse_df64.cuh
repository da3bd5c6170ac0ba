// hse_df64.cuh -- double-float ("df64") arithmetic on the FP32 pipe.
//
// A df64 value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  Sums and products use the
// error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the
// FMA two-product; the addition is the cheap ("sloppy") variant that adds the
// low parts without their own error term, whose error is bounded relative to
// |a| + |b| (enough for transforms, whose error analysis is norm-wise).
// Reference: Y. Hida, X. S. Li, D. H. Bailey, "Library for double-double and
// quad-double arithmetic" (2007), and A. Thall, "Extended-precision
// floating-point numbers for GPU computation" (2006).
//
// GB300 issues 128 FP32 lanes per SM and clock against 2 FP64 instructions, so
// a df64 operation of 5-11 FP32 instructions is several times cheaper than its
// FP64 counterpart; double <-> float conversions run at the FP64 rate and are
// kept to the edges of a computation.
#pragma once
#include <cuda_runtime.h>

namespace hse {

struct __align__(8) df {
  float hi, lo;
  df() = default;  // trivial: usable in __shared__ arrays
  __device__ __forceinline__ df(float h, float l) : hi(h), lo(l) {}
  // exact for integers of magnitude < 2^24
  __device__ __forceinline__ df(int i) : hi((float)i), lo(0.f) {}
  // rounds to ~48 bits (FP64-pipe conversions)
  __device__ __forceinline__ df(double d) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
  }
  __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
};

// conversions between the grid element types (double, float, df)
__device__ __forceinline__ float head32(double v) { return (float)v; }
__device__ __forceinline__ float head32(float v) { return v; }
__device__ __forceinline__ float head32(df v) { return v.hi; }
__device__ __forceinline__ double to64(double v) { return v; }
__device__ __forceinline__ double to64(float v) { return (double)v; }
__device__ __forceinline__ double to64(df v) { return v.to_double(); }
template <typename T> __device__ __forceinline__ T from32(float f) { return (T)f; }
template <> __device__ __forceinline__ df from32<df>(float f) { return df(f, 0.f); }

// s + e == a + b exactly, provided |a| >= |b| or a == 0
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df operator+(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s, e);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// product with a float that is exact in df64 (an integer or a power of two)
__device__ __forceinline__ df operator*(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = fmaf(a.hi, b, -p);
  e = fmaf(a.lo, b, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df operator*(float b, df a) { return a * b; }
__device__ __forceinline__ df operator*(df a, int i) { return a * (float)i; }
__device__ __forceinline__ df operator*(int i, df a) { return a * (float)i; }
// a b + c (the real-space pair terms are written with fma(); for df64 they
// take this double-float multiply-add).  The float and double overloads stay
// visible inside the namespace.
using ::fma;
using ::fmaf;
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return c + df(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator-=(df& a, df b) { return a = a - b; }

// Unnormalised forms for intermediate results inside a computation: the pair
// (s, e) still sums to the value with the same error bound, but |e| may exceed
// ulp(s) / 2 by a few units.  Every df64 operation above accepts such inputs;
// df_norm restores the invariant before a value is stored.
__device__ __forceinline__ df df_add_raw(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_sub_raw(df a, df b) { return df_add_raw(a, -b); }
__device__ __forceinline__ df df_mul_raw(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  return df(p, fmaf(a.lo, b.hi, e));
}
__device__ __forceinline__ df df_norm(df a) { return df_fast_two_sum(a.hi, a.lo); }

// a b - c d with one rounding-error-free difference of the leading products
// (16 FP32 operations against 25 for two products and a sum), unnormalised
__device__ __forceinline__ df df_dot2_raw(df a, df b, df c, df d) {
  const float p = __fmul_rn(a.hi, b.hi), q = __fmul_rn(c.hi, d.hi);
  const float e1 = fmaf(a.hi, b.hi, -p), e2 = fmaf(c.hi, d.hi, -q);
  const float s = __fsub_rn(p, q);
  const float bb = __fsub_rn(s, p);
  float e = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(-q, bb));
  e = __fadd_rn(e, __fsub_rn(e1, e2));
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  e = fmaf(-c.hi, d.lo, e);
  e = fmaf(-c.lo, d.hi, e);
  return df(s, e);
}

// multiply-accumulate acc + a b and the product a b in the grid element type:
// FMA for double and float, an unnormalised product added with renormalisation
// for df64 (products that only feed a sum need no renormalisation of their own)
__device__ __forceinline__ double mac(double acc, double a, double b) { return fma(a, b, acc); }
__device__ __forceinline__ float mac(float acc, float a, float b) { return fmaf(a, b, acc); }
__device__ __forceinline__ df mac(df acc, df a, df b) { return acc + df_mul_raw(a, b); }
__device__ __forceinline__ double mulr(double a, double b) { return a * b; }
__device__ __forceinline__ float mulr(float a, float b) { return a * b; }
__device__ __forceinline__ df mulr(df a, df b) { return df_mul_raw(a, b); }

// complex df64, laid out like a complex double (16 bytes)
struct __align__(16) cdf {
  df x, y;
};

__device__ __forceinline__ cdf cdf_make(df x, df y) {
  cdf r;
  r.x = x;
  r.y = y;
  return r;
}
__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return cdf_make(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return cdf_make(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cdf operator*(cdf a, cdf b) {
  return cdf_make(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ cdf operator*(df s, cdf a) { return cdf_make(s * a.x, s * a.y); }
__device__ __forceinline__ cdf conj(cdf a) { return cdf_make(a.x, -a.y); }
__device__ __forceinline__ cdf add_raw(cdf a, cdf b) { return cdf_make(df_add_raw(a.x, b.x), df_add_raw(a.y, b.y)); }
__device__ __forceinline__ cdf sub_raw(cdf a, cdf b) { return cdf_make(df_sub_raw(a.x, b.x), df_sub_raw(a.y, b.y)); }
__device__ __forceinline__ cdf scale_raw(df s, cdf a) { return cdf_make(df_mul_raw(s, a.x), df_mul_raw(s, a.y)); }
// a w (w = wr + i wi), unnormalised
__device__ __forceinline__ cdf mul_raw(cdf a, cdf w) {
  return cdf_make(df_dot2_raw(a.x, w.x, a.y, w.y), df_dot2_raw(a.x, w.y, -a.y, w.x));
}
__device__ __forceinline__ cdf norm(cdf a) { return cdf_make(df_norm(a.x), df_norm(a.y)); }
// multiply by -i (forward transforms) or +i (inverse)
template <bool FWD>
__device__ __forceinline__ cdf mul_mi(cdf a) {
  return FWD ? cdf_make(a.y, -a.x) : cdf_make(-a.y, a.x);
}

__device__ __forceinline__ cdf ld_cdf(const float4* p) {
  const float4 v = *p;
  return cdf_make(df(v.x, v.y), df(v.z, v.w));
}
__device__ __forceinline__ cdf ldg_cdf(const float4* p) {
  const float4 v = __ldg(p);
  return cdf_make(df(v.x, v.y), df(v.z, v.w));
}
__device__ __forceinline__ void st_cdf(float4* p, cdf a) { *p = make_float4(a.x.hi, a.x.lo, a.y.hi, a.y.lo); }

}  // namespace hse
