// Double-float arithmetic ("df64"): a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi)/2, giving a 48-bit significand (relative
// rounding error about 2^-48 per operation) computed on the FP32 pipe.  On GB300
// the FP32 pipe is about 64x wider than the FP64 pipe, so FP64-grade
// recurrences run faster this way.  The operations follow the classical
// error-free transformations: Knuth's TwoSum and the FMA-based TwoProduct
// (Dekker 1971; Hida, Li & Bailey, "Library for double-double and quad-double
// arithmetic", 2001), with one Newton correction for division and square root.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tadmm {

// keep the float/double fma overloads visible next to the df64 one
using ::fma;

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df64(int v) : hi((float)v), lo((float)(v - (int)(float)v)) {}
  __host__ __device__ df64(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ df64(double v) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 quick_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  return quick_two_sum(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
// a * b + c with one renormalization
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = p + c.hi;
  const float v = s - p;
  float t = (p - (s - v)) + (c.hi - v);
  t += e + c.lo;
  return quick_two_sum(s, t);
}
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float q1 = a.hi / b.hi;
  const df64 r = a - b * df64(q1);
  const float q2 = r.hi / b.hi;
  const df64 r2 = r - b * df64(q2);
  const float q3 = r2.hi / b.hi;
  return quick_two_sum(q1, q2) + df64(q3);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
__device__ __forceinline__ df64& operator/=(df64& a, df64 b) { return a = a / b; }

__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a) && a.hi == a.hi && b.hi == b.hi; }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return b <= a; }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

__device__ __forceinline__ df64 fabs_(df64 v) { return v.hi < 0.0f ? -v : v; }
__device__ __forceinline__ df64 sqrt_(df64 a) {
  if (!(a.hi > 0.0f)) return df64(sqrtf(a.hi), 0.0f);
  const float s = sqrtf(a.hi);
  const df64 e = a - df64(s) * df64(s);
  return quick_two_sum(s, e.hi / (2.0f * s));
}
__device__ __forceinline__ bool finite_(df64 v) { return isfinite(v.hi) && isfinite(v.lo); }
__device__ __forceinline__ bool sign_set(df64 v) { return __float_as_int(v.hi) < 0; }

// Order-preserving 32-bit key of a float and its inverse.
__device__ __forceinline__ uint32_t f32_key(float x) {
  const int b = __float_as_int(x);
  return (uint32_t)(b ^ ((b >> 31) | (int)0x80000000u));
}
__device__ __forceinline__ float f32_unkey(uint32_t k) {
  const uint32_t b = (k & 0x80000000u) ? (k ^ 0x80000000u) : ~k;
  return __int_as_float((int)b);
}
// A normalized df64 orders lexicographically by (hi, lo).
__device__ __forceinline__ unsigned long long mono_key(df64 v) {
  return ((unsigned long long)f32_key(v.hi) << 32) | f32_key(v.lo);
}
__device__ __forceinline__ unsigned long long abs_bits(df64 v) {
  const df64 a = fabs_(v);
  return ((unsigned long long)(uint32_t)__float_as_int(a.hi) << 32) | f32_key(a.lo);
}
__device__ __forceinline__ unsigned long long ord_bits(df64 v) { return abs_bits(v); }
// NaN test on an abs_bits key (the high word carries |hi|).
__device__ __forceinline__ bool nan_key(unsigned long long ab, df64) { return (ab >> 32) > 0x7F800000ull; }
__device__ __forceinline__ df64 from_bits(unsigned long long b, df64) {
  return df64(__int_as_float((int)(uint32_t)(b >> 32)), f32_unkey((uint32_t)b));
}

}  // namespace tadmm
