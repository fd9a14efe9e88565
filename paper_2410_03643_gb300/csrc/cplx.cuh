// Complex helpers on double2 / float2 (x = real part, y = imaginary part).
#pragma once
#include <cuda_runtime.h>

namespace rfnse {

template <typename R> struct cvec;
template <> struct cvec<double> {
  using type = double2;
  static __host__ __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <> struct cvec<float> {
  using type = float2;
  static __host__ __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <typename R> using cv = typename cvec<R>::type;
// the real type of a complex type
template <typename V> struct creal {
  using type = decltype(V().x);
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
// a * b
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// i * a and -i * a
__device__ __forceinline__ double2 cmul_i(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ float2 cmul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ double2 cmul_mi(double2 a) { return make_double2(a.y, -a.x); }
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// Packed float pairs (sm_100 family): one instruction applies the same FP32 operation, rounded to
// nearest on its own (never contracted), to both halves; per component the result is that of the
// scalar _rn operation.
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 f2_bcast(float v) { return make_float2(v, v); }

// conversions between storage and compute precision
template <typename R> __device__ __forceinline__ cv<R> to_c(double2 v);
template <> __device__ __forceinline__ double2 to_c<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_c<float>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <typename R> __device__ __forceinline__ cv<R> to_c(float2 v);
template <> __device__ __forceinline__ double2 to_c<double>(float2 v) { return make_double2(v.x, v.y); }
template <> __device__ __forceinline__ float2 to_c<float>(float2 v) { return v; }

template <typename S> struct store_of;
template <> struct store_of<double> { using type = double2; };
template <> struct store_of<float> { using type = float2; };

__device__ __forceinline__ void st_c(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void st_c(double2* p, float2 v) { *p = make_double2(v.x, v.y); }
__device__ __forceinline__ void st_c(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void st_c(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

}  // namespace rfnse
