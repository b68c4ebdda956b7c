// Host check of the double-float split of a double (df64.cuh): hi = fl(x) and
// lo = fl(x - hi), rounded to nearest even, must come out bit for bit as from FP64 arithmetic,
// whichever path (integer and FP32, or FP64) the constructor takes. Exit status 0 when all
// values agree.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../../paper_1404_3773_gb300/csrc/df64.cuh"

static bool same(double x) {
  const cs::df64 d(x);
  const float h = (float)x;
  const float l = (float)(x - (double)h);
  uint32_t a, b, c, e;
  std::memcpy(&a, &d.hi, 4);
  std::memcpy(&b, &h, 4);
  std::memcpy(&c, &d.lo, 4);
  std::memcpy(&e, &l, 4);
  if (a == b && c == e) return true;
  std::printf("mismatch x = %.17g: hi %a vs %a, lo %a vs %a\n", x, d.hi, h, d.lo, l);
  return false;
}

int main() {
  std::mt19937_64 g(20240611);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  long n = 0, bad = 0;
  // magnitudes 2^-130 .. 2^130: both sides of the integer path's range
  for (int i = 0; i < 400000; ++i, ++n) bad += !same(std::ldexp(u(g), (int)(g() % 261) - 130));
  // the 29 bits below hi at a tie, just below and just above it (rounding and carries)
  const uint64_t low[] = {0x10000000ull, 0x0FFFFFFFull, 0x10000001ull, 0x1FFFFFFFull, 0ull};
  for (int i = 0; i < 100000; ++i, ++n) {
    uint64_t b = (g() & ~0x1FFFFFFFull) | low[g() % 5];
    double x;
    std::memcpy(&x, &b, 8);
    if (!std::isfinite(x)) x = 1.0;
    bad += !same(x);
  }
  const double edge[] = {0.0, -0.0, 1.0, -1.0, 0.1, -1.0 / 3.0, 1e-30, -1e-22, 1e38, -3e38,
                         1e-300, 1e300, std::ldexp(1.0, -74), std::ldexp(1.0, -75),
                         std::ldexp(1.0, 125), std::ldexp(1.0, 126),
                         std::ldexp(1.0 - std::ldexp(1.0, -53), 125),
                         std::ldexp(1.0 - std::ldexp(1.0, -53), 126)};
  for (double x : edge) {
    ++n;
    bad += !same(x);
  }
  std::printf("%ld values, %ld mismatches\n", n, bad);
  return bad != 0;
}
