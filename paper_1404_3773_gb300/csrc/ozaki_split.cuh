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
  int n = 0;
  while (v) {
    ++n;
    v >>= 1;
  }
  return n;
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

// One entry of C = A^T B from the exact slice products S[k * s + l] = a_k^T b_l of its column
// pair (column exponents E of A, F of B): the sum over the pairs with k + l <= s - 1, smallest
// terms first (k + l from s - 1 down to 0, k ascending within), in FP64. Each term
// 2^(E + F - 2 (beta - 1) - (k + l) beta) S is exact; the additions are the only roundings.
// Requires |S| < 2^53 and the exponents inside the normal FP64 range.
__host__ __device__ inline double oz_combine(const int64_t* S, int E, int F, int beta, int s) {
  double c = 0.0;
  for (int m = s - 1; m >= 0; --m)
    for (int k = 0; k <= m; ++k) {
      const int l = m - k;
      const double term = (double)S[k * s + l] * oz_pow2(E + F - 2 * (beta - 1) - m * beta);
      c = c + term;
    }
  return c;
}

}  // namespace cs
