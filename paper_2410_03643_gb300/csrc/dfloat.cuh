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

// complex double-float, stored as the pairs hi = (re.hi, im.hi) and lo = (re.lo, im.lo), so that the
// real and imaginary parts go through every step of an operation together as packed pairs: the same
// operations, in the same order, as the scalar double-float arithmetic above on each part.
struct cdf {
  float2 hi, lo;
};
template <> struct cvec<dfl> {
  using type = cdf;
  static __host__ __device__ __forceinline__ cdf make(dfl a, dfl b) {
    return cdf{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
  }
};
template <> struct creal<cdf> {
  using type = dfl;
};

// TwoSum and FastTwoSum on pairs; a + b and a - b of double-float pairs (operator+ above per part)
__device__ __forceinline__ cdf cadd(cdf a, cdf b) {
  const float2 s = f2_add(a.hi, b.hi);
  const float2 bb = f2_sub(s, a.hi);
  const float2 e = f2_add(f2_sub(a.hi, f2_sub(s, bb)), f2_sub(b.hi, bb));
  const float2 t = f2_add(e, f2_add(a.lo, b.lo));
  const float2 s2 = f2_add(s, t);
  return cdf{s2, f2_sub(t, f2_sub(s2, s))};
}
__device__ __forceinline__ cdf csub(cdf a, cdf b) {  // a + (-b): -b - bb = -(b + bb)
  const float2 s = f2_sub(a.hi, b.hi);
  const float2 bb = f2_sub(s, a.hi);
  const float2 e = f2_sub(f2_sub(a.hi, f2_sub(s, bb)), f2_add(b.hi, bb));
  const float2 t = f2_add(e, f2_sub(a.lo, b.lo));
  const float2 s2 = f2_add(s, t);
  return cdf{s2, f2_sub(t, f2_sub(s2, s))};
}
// (x.hi + x.lo) times each component of the pair (bh + bl): TwoProd by FMA with the cross terms, then
// FastTwoSum (operator* above per part).  With q = fl(-x.hi bh) = -p exactly: e = fma(x.hi, bh, q),
// s = fl(e - q) = fl(p + e), e' = e - (s + q) = e - (s - p).
__device__ __forceinline__ cdf df_scale_pair(float xh, float xl, float2 bh, float2 bl) {
  const float2 xh2 = f2_bcast(xh);
  const float2 q = f2_mul(f2_bcast(-xh), bh);
  float2 e = f2_fma(xh2, bh, q);
  e = f2_fma(xh2, bl, e);
  e = f2_fma(f2_bcast(xl), bh, e);
  const float2 s = f2_sub(e, q);
  return cdf{s, f2_sub(e, f2_add(s, q))};
}
__device__ __forceinline__ cdf cneg(cdf a) {
  return cdf{make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y)};
}
// a b = (a.re b.re - a.im b.im, a.re b.im + a.im b.re): the pairs a.re (b.re, b.im) and
// a.im (b.im, b.re), then one pair addition with the first component of the second negated
__device__ __forceinline__ cdf cmul(cdf a, cdf b) {
  const cdf x = df_scale_pair(a.hi.x, a.lo.x, b.hi, b.lo);
  const cdf y = df_scale_pair(a.hi.y, a.lo.y, make_float2(b.hi.y, b.hi.x), make_float2(b.lo.y, b.lo.x));
  return cadd(x, cdf{make_float2(-y.hi.x, y.hi.y), make_float2(-y.lo.x, y.lo.y)});
}
__device__ __forceinline__ cdf cscale(cdf a, dfl s) {  // (a.re s, a.im s)
  const float2 sh = f2_bcast(s.hi);
  const float2 q = f2_mul(make_float2(-a.hi.x, -a.hi.y), sh);
  float2 e = f2_fma(a.hi, sh, q);
  e = f2_fma(a.hi, f2_bcast(s.lo), e);
  e = f2_fma(a.lo, sh, e);
  const float2 r = f2_sub(e, q);
  return cdf{r, f2_sub(e, f2_add(r, q))};
}
__device__ __forceinline__ cdf cmul_i(cdf a) {
  return cdf{make_float2(-a.hi.y, a.hi.x), make_float2(-a.lo.y, a.lo.x)};
}
__device__ __forceinline__ cdf cmul_mi(cdf a) {
  return cdf{make_float2(a.hi.y, -a.hi.x), make_float2(a.lo.y, -a.lo.x)};
}
__device__ __forceinline__ cdf cconj(cdf a) {
  return cdf{make_float2(a.hi.x, -a.hi.y), make_float2(a.lo.x, -a.lo.y)};
}
__device__ __forceinline__ cdf cdf_from(double2 v) { return cvec<dfl>::make(df_split(v.x), df_split(v.y)); }
// storage of a complex double-float as (re.hi, im.hi, re.lo, im.lo)
__device__ __forceinline__ cdf cdf_ld(float4 q) { return cdf{make_float2(q.x, q.y), make_float2(q.z, q.w)}; }
__device__ __forceinline__ float4 cdf_st(cdf v) { return make_float4(v.hi.x, v.hi.y, v.lo.x, v.lo.y); }
__device__ __forceinline__ double2 cdf_to(cdf v) {
  return make_double2(df_to_double(dfl(v.hi.x, v.lo.x)), df_to_double(dfl(v.hi.y, v.lo.y)));
}

}  // namespace rfnse
