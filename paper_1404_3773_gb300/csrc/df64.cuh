// Double-float ("df64") arithmetic on the FP32 pipe (internal). A value is the unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits. Built from
// the error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2): two_sum gives
// a + b = s + e exactly; with a fused multiply-add, a * b - p is exact as fmaf(a, b, -p).
// On GB300 the FP64 pipe retires 1/64 of the FP32 rate, so a df64 multiply-add (about 15
// FP32 instructions) is several times faster than a native FP64 one while keeping relative
// errors near 2^-44 of the summed magnitudes, far inside the 1e-11 parity bar of H X.
// The exponent range is FP32's; the values of this method (tables of order 1 to 1e3, states
// of order 1) stay far from it. Requires IEEE FP32 semantics (no fast-math contraction or
// flush-to-zero of the lo parts).
#pragma once

#include <cuda_runtime.h>

namespace cs {

// the df64 overload of fma below must not hide the FP64/FP32 ones for unqualified calls
using ::fma;

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // exact split of a double into hi + lo (lo carries the next 24 bits)
  __host__ __device__ df64(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ df64(int x) : df64((double)x) {}
  __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (no condition on the magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  float h, l;
  quick_two_sum(s, e, h, l);
  return df64(h, l);
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float h, l;
  quick_two_sum(p, e, h, l);
  return df64(h, l);
}
// a * b + c, the product kept unrounded (p + e) until it meets c
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t += e + c.lo;
  float h, l;
  quick_two_sum(s, t, h, l);
  return df64(h, l);
}
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }

}  // namespace cs
