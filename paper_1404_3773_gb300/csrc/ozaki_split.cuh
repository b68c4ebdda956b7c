// Integer slices of FP64 values for exact low-precision matrix products (internal): the
// error-free splitting of Ozaki, Ogita, Oishi and Rump (2012) in its integer-slice form, for
// the FP64 Gram matrices and rotations of the dense steps (Sec. 3.2).
//
// A column with E = ceil(log2 max|x|) is cut into s slices of beta bits: the unit of slice k
// (0-based) is u_k = 2^(E - (beta - 1) - k beta), and a_k = rne(r_k / u_k) with r_0 = x,
// r_{k+1} = r_k - a_k u_k (rne: round to nearest, ties to even). Every a_k is an integer with
// |a_k| <= 2^(beta - 1), exactly a BF16 value for beta <= 9.
//
// The digits are computed here from the bits of x with integer arithmetic only (GB300's FP64
// pipe runs at 1/64 of the FP32 rate). The residual is held in sign-magnitude as an integer
// count of half last-units, delta = u_{s-1} / 2, plus a sticky flag for any bits below delta:
// that is enough to decide every rounding, ties included, exactly as FP64 arithmetic on the
// exact residuals would.
#pragma once

#include <cstdint>
#include <cstring>

namespace cs {

__host__ __device__ inline uint64_t oz_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

// |x| = M 2^q with M an integer below 2^53 (0 for x = 0)
__host__ __device__ inline void oz_decompose(double x, uint64_t& M, int& q) {
  const uint64_t b = oz_bits(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const uint64_t f = b & 0xFFFFFFFFFFFFFull;
  if (e == 0) {  // zero or subnormal
    M = f;
    q = -1074;
  } else {
    M = f | (1ull << 52);
    q = e - 1075;
  }
}

__host__ __device__ inline int oz_bit_length(uint64_t v) {
#ifdef __CUDA_ARCH__
  return 64 - __clzll((long long)v);
#else
  int n = 0;
  while (v) {
    ++n;
    v >>= 1;
  }
  return n;
#endif
}

// ceil(log2 m) for m = max |x| of a column (m > 0); 0 for m = 0
__host__ __device__ inline int oz_exponent(double m) {
  uint64_t M;
  int q;
  oz_decompose(m, M, q);
  if (M == 0) return 0;
  const int n = oz_bit_length(M);  // m = M 2^q, 2^(n-1) <= M < 2^n
  const bool pow2 = (M & (M - 1)) == 0;
  return q + (pow2 ? n - 1 : n);
}

// The s digits of x for a column of exponent E (|x| <= 2^E). a[k] receives a_k.
// Requires 2 <= beta <= 30 and s beta <= 62.
__host__ __device__ inline void oz_slices(double x, int E, int beta, int s, int* a) {
  uint64_t M;
  int q;
  oz_decompose(x, M, q);
  const bool neg = (oz_bits(x) >> 63) != 0;
  // residual |r| = mag delta + (sticky ? something in (0, delta) : 0), delta = 2^(t_last - 1)
  const int t_last = E - (beta - 1) - (s - 1) * beta;
  const int shift = q - (t_last - 1);
  uint64_t mag;
  bool sticky;
  if (M == 0) {
    mag = 0;
    sticky = false;
  } else if (shift >= 0) {
    mag = M << shift;  // |x| / delta <= 2^(s beta) (|x| <= 2^E)
    sticky = false;
  } else if (shift > -64) {
    mag = M >> (-shift);
    sticky = (M & ((1ull << (-shift)) - 1)) != 0;
  } else {
    mag = 0;
    sticky = true;
  }
  bool rneg = neg;  // sign of the residual
  for (int k = 0; k < s; ++k) {
    const int sh = (s - 1 - k) * beta + 1;  // u_k = 2^sh delta
    const uint64_t U = 1ull << sh, half = U >> 1;
    uint64_t qd = mag >> sh;
    const uint64_t rem = mag & (U - 1);
    const bool up = rem > half || (rem == half && (sticky || (qd & 1)));
    if (up) {
      ++qd;
      // new residual: qd U - |r|, with the opposite sign
      const uint64_t top = qd << sh;  // >= mag
      if (sticky) {
        mag = top - mag - 1;  // (top - mag) delta - eps = (top - mag - 1) delta + (delta - eps)
      } else {
        mag = top - mag;
      }
      a[k] = rneg ? -(int)qd : (int)qd;
      rneg = !rneg;
    } else {
      mag = rem;  // |r| - qd U, same sign
      a[k] = rneg ? -(int)qd : (int)qd;
    }
  }
}

// 2^e as a double (|e| <= 1022)
__host__ __device__ inline double oz_pow2(int e) {
  const uint64_t b = (uint64_t)(e + 1023) << 52;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, sizeof v);
  return v;
#endif
}

// A signed 128-bit integer as two's complement (hi, lo), enough for the exact sums below.
struct OzI128 {
  int64_t hi = 0;
  uint64_t lo = 0;
};

// acc += v * 2^sh  (0 <= sh < 64, |v| 2^sh < 2^126)
__host__ __device__ inline void oz_add_shifted(OzI128& acc, int64_t v, int sh) {
  const uint64_t lo = (uint64_t)v << sh;
  const int64_t hi = sh == 0 ? (v < 0 ? -1 : 0) : (v >> (64 - sh));  // arithmetic shift
  const uint64_t nlo = acc.lo + lo;
  acc.hi = acc.hi + hi + (nlo < acc.lo ? 1 : 0);
  acc.lo = nlo;
}

// The integer acc rounded to the nearest double (ties to even), times 2^e (the result must stay
// in the normal range; e only shifts the exponent).
__host__ __device__ inline double oz_round_i128(OzI128 acc, int e) {
  const bool neg = acc.hi < 0;
  uint64_t hi = (uint64_t)acc.hi, lo = acc.lo;
  if (neg) {  // magnitude: two's complement negation
    lo = ~lo + 1;
    hi = ~hi + (lo == 0 ? 1 : 0);
  }
  if (hi == 0 && lo == 0) return 0.0;
  // top bit position p of the 128-bit magnitude
  const int p = hi ? 64 + oz_bit_length(hi) - 1 : oz_bit_length(lo) - 1;
  uint64_t m;
  int ex;  // value = m 2^ex, m < 2^53
  if (p <= 52) {
    m = lo;
    ex = 0;
  } else {
    const int sh = p - 52;  // bits below the kept 53
    // m = magnitude >> sh; rem = magnitude mod 2^sh (as a comparison against half)
    if (sh >= 64) {
      m = hi >> (sh - 64);
    } else {
      m = (lo >> sh) | (sh ? (hi << (64 - sh)) : 0);
    }
    // round bit and sticky bits
    const int rb = sh - 1;  // position of the round bit
    const bool round_bit =
        rb >= 64 ? ((hi >> (rb - 64)) & 1) != 0 : ((lo >> rb) & 1) != 0;
    bool sticky;
    if (rb >= 64) {
      sticky = lo != 0 || (rb - 64 > 0 && (hi & ((1ull << (rb - 64)) - 1)) != 0);
    } else {
      sticky = rb > 0 && (lo & ((1ull << rb) - 1)) != 0;
    }
    if (round_bit && (sticky || (m & 1))) ++m;
    ex = sh;
    if (m == (1ull << 53)) {  // carried into a new bit
      m >>= 1;
      ++ex;
    }
  }
  const double v = (double)m * oz_pow2(ex + e);  // m < 2^53: exact; times a power of two
  return neg ? -v : v;
}

// One entry of C = A^T B from the exact diagonal sums D[t] = sum_{k + l = t} a_k^T b_l of its
// column pair (t = 0 .. s - 1; column exponents E of A, F of B): the exact value
// sum_t D[t] 2^(E + F - 2 (beta - 1) - t beta) rounded once to FP64 (nearest, ties to even).
// Requires (s - 1) beta <= 63 and |D[t]| 2^((s - 1 - t) beta) < 2^125 (no 128-bit overflow).
__host__ __device__ inline double oz_combine(const int64_t* D, int E, int F, int beta, int s) {
  OzI128 acc;
  for (int t = 0; t < s; ++t) oz_add_shifted(acc, D[t], (s - 1 - t) * beta);
  return oz_round_i128(acc, E + F - 2 * (beta - 1) - (s - 1) * beta);
}

}  // namespace cs
