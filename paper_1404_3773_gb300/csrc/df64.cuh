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

#include <cstdint>
#include <cstring>

namespace cs {

__host__ __device__ inline uint64_t df64_bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}
__host__ __device__ inline float df64_float_of(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  std::memcpy(&f, &b, sizeof f);
  return f;
#endif
}

// the df64 overload of fma below must not hide the FP64/FP32 ones for unqualified calls
using ::fma;

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // split of a double into hi = fl(x) and lo = fl(x - hi), both rounded to nearest even (lo
  // carries the next 24 bits). Where hi and the unit of x's last bit are normal floats
  // (2^-74 <= |x| < 2^126) this is done on the integer and FP32 pipes from x's bits: hi is
  // x's top 24 significant bits rounded to nearest even, and x - hi is the remaining 29-bit
  // integer (minus 2^29 when hi rounded up) times 2^(e - 1075), converted with one rounding.
  // Elsewhere the same values come from FP64 arithmetic, which GB300 runs at 1/64 rate.
  __host__ __device__ df64(double x) {
    const uint64_t b = df64_bits_of(x);
    const int e = (int)((b >> 52) & 0x7FF);  // biased exponent
    if (e >= 949 && e <= 1148) {
      const uint64_t mant = b & 0xFFFFFFFFFFFFFull;
      const uint32_t r = (uint32_t)(mant & 0x1FFFFFFFu);  // the 29 bits below hi
      uint32_t hb = ((uint32_t)(b >> 63) << 31) | ((uint32_t)(e - 896) << 23) |
                    (uint32_t)(mant >> 29);
      const bool up = r > 0x10000000u || (r == 0x10000000u && (hb & 1u));
      hb += up ? 1u : 0u;  // a carry moves into the exponent, as rounding does
      int res = (int)r - (up ? 0x20000000 : 0);  // |res| <= 2^28
      if (b >> 63) res = -res;                    // signed residual; zero stays +0
      const float scale = df64_float_of((uint32_t)(e - 1075 + 127) << 23);  // 2^(e - 1075)
      hi = df64_float_of(hb);
      lo = (float)res * scale;
    } else {
      hi = (float)x;
      lo = (float)(x - (double)(float)x);
    }
  }
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

// Accumulator of a sum of df64 products without the per-step renormalisation of fma above:
// each step adds the exact rounded product p = a.hi b.hi to hi by two_sum (exact), and the
// product's error terms and two_sum's error to lo; hi + lo is renormalised once, when read.
// 12 FP32 instructions per multiply-add instead of 15. lo stays small against hi for the short
// sums it is used for (at most a few hundred terms of table-times-value products), so the
// result keeps the df64 accuracy.
struct df64acc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add_prod(df64 a, df64 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo += err + e;
  }
  __device__ __forceinline__ df64 value() const {
    float s, e;
    two_sum(hi, lo, s, e);
    return df64(s, e);
  }
};
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }

// Multiply-add accumulator over an arithmetic type: a fused multiply-add for float and double,
// df64acc for df64 (one renormalisation when read).
template <typename C>
struct MacAcc {
  C v = C(0);
  __device__ __forceinline__ void set(C x) { v = x; }
  __device__ __forceinline__ void add_prod(C a, C b) { v = fma(a, b, v); }
  __device__ __forceinline__ C value() const { return v; }
};
template <>
struct MacAcc<df64> {
  df64acc a;
  __device__ __forceinline__ void set(df64 x) {
    a.hi = x.hi;
    a.lo = x.lo;
  }
  __device__ __forceinline__ void add_prod(df64 x, df64 y) { a.add_prod(x, y); }
  __device__ __forceinline__ df64 value() const { return a.value(); }
};

}  // namespace cs
