// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits.  Built from two error-free transformations:
//   TwoSum (Knuth):   s = fl(a + b) and e = (a - (s - bb)) + (b - bb), bb = s - a, give a + b = s + e;
//   TwoProd with FMA: p = fl(a b) and e = fma(a, b, -p) give a b = p + e exactly.
// Addition adds the low parts and renormalises with FastTwoSum; multiplication keeps the cross terms
// hi*lo (the lo*lo term is below the format's precision).  Relative error of one operation is a few
// units of 2^-48 (for sums of values of opposite sign the bound is relative to |a| + |b|), enough for
// an FFT whose normwise error is what matters.
//
// Used for the Toeplitz products of the mixed form's FP64 residual: GB300 issues FP32 FMA 61 times
// faster than FP64 FMA, and a double-float FFT costs roughly eight times the FP32 instructions.
// The compiler must not reassociate these operations (no fast-math).
#pragma once
#include "cplx.cuh"

namespace rfnse {

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  // from FP64: hi = fl32(x), lo = fl32(x - hi) (exact difference in FP64)
  __host__ __device__ dfl(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

// The additions and the leading product use the _rn intrinsics, which the compiler never contracts into
// a fused multiply-add: the transformations rely on every one of them being rounded on its own.
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e);
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return dfl(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// Conversions with few FP64 instructions (GB300's FP64 pipe is the scarce one).  float -> double of a
// normal float is exact bit manipulation (sign, rebiased exponent, significand shifted left by 29);
// zeros, subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double df_f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e8 = (b >> 23) & 0xffu;
  if (e8 == 0u || e8 == 0xffu) return (double)f;
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(e8 + (1023u - 127u)) << 52) |
                               ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}
// double -> double-float: hi = x with its significand truncated to 24 bits (integer work when x is in
// the normal float range), lo = fl32(x - hi) (one exact FP64 subtraction and one conversion).
__device__ __forceinline__ dfl df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
  if (e >= 255) return dfl((float)x, 0.0f);  // beyond the float range: +-inf (or NaN) in hi alone
  if (e <= 0) return dfl(x);                 // zero and tiny values: the FP64 path
  const double hd = __longlong_as_double((long long)(b & 0xFFFFFFFFE0000000ull));
  const unsigned hb = (unsigned)(b >> 32 & 0x80000000ull) | ((unsigned)e << 23) | (unsigned)((b >> 29) & 0x7fffffull);
  return dfl(__uint_as_float(hb), __double2float_rn(x - hd));
}
__device__ __forceinline__ double df_to_double(dfl a) { return df_f2d(a.hi) + df_f2d(a.lo); }

// complex double-float
struct cdf {
  dfl x, y;
};
template <> struct cvec<dfl> {
  using type = cdf;
  static __host__ __device__ __forceinline__ cdf make(dfl a, dfl b) { return cdf{a, b}; }
};

__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return cdf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return cdf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cdf cneg(cdf a) { return cdf{-a.x, -a.y}; }
__device__ __forceinline__ cdf cmul(cdf a, cdf b) { return cdf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cdf cscale(cdf a, dfl s) { return cdf{a.x * s, a.y * s}; }
__device__ __forceinline__ cdf cmul_i(cdf a) { return cdf{-a.y, a.x}; }
__device__ __forceinline__ cdf cmul_mi(cdf a) { return cdf{a.y, -a.x}; }
__device__ __forceinline__ cdf cdf_from(double2 v) { return cdf{df_split(v.x), df_split(v.y)}; }
// storage of a complex double-float as (re.hi, re.lo, im.hi, im.lo)
__device__ __forceinline__ cdf cdf_ld(float4 q) { return cdf{dfl(q.x, q.y), dfl(q.z, q.w)}; }
__device__ __forceinline__ float4 cdf_st(cdf v) { return make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo); }
__device__ __forceinline__ double2 cdf_to(cdf v) { return make_double2(df_to_double(v.x), df_to_double(v.y)); }

}  // namespace rfnse
