// Host emulation of the tensor-core data flow for C = A^T B from integer slices
// (ozaki_split.cuh): per-column exponents from a max pre-pass; the split; per chunk of
// `chunk` rows and per diagonal k + l = t, a partial sum that one FP32 tensor-memory
// accumulator of a CTA must hold exactly (checked: the sum of the magnitudes of its products
// stays within 2^24, which bounds every running sum in any order of addition); the
// partials added in 64-bit integers; oz_combine. The result is compared with the oracle's C
// bit for bit.
// Input file: int32 d, na, nb, beta, s, chunk; A (d x na, FP64, column-major); B (d x nb);
// the oracle's C (na x nb, row-major). Exit status 0 on agreement.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../paper_1404_3773_gb300/csrc/ozaki_split.cuh"

static void slices(const std::vector<double>& X, int d, int n, int beta, int s,
                   std::vector<int>& E, std::vector<int>& a) {
  E.assign(n, 0);
  a.assign((size_t)s * d * n, 0);
  std::vector<int> dig(s);
  for (int j = 0; j < n; ++j) {
    double m = 0.0;
    for (int r = 0; r < d; ++r) m = std::fmax(m, std::fabs(X[(size_t)j * d + r]));
    E[j] = cs::oz_exponent(m);
    for (int r = 0; r < d; ++r) {
      cs::oz_slices(X[(size_t)j * d + r], E[j], beta, s, dig.data());
      for (int k = 0; k < s; ++k) a[((size_t)k * n + j) * d + r] = dig[k];
    }
  }
}

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t h[6];
  if (std::fread(h, 4, 6, f) != 6) return 2;
  const int d = h[0], na = h[1], nb = h[2], beta = h[3], s = h[4], chunk = h[5];
  std::vector<double> A((size_t)d * na), B((size_t)d * nb), C((size_t)na * nb);
  if (std::fread(A.data(), 8, A.size(), f) != A.size()) return 2;
  if (std::fread(B.data(), 8, B.size(), f) != B.size()) return 2;
  if (std::fread(C.data(), 8, C.size(), f) != C.size()) return 2;
  std::fclose(f);
  std::vector<int> EA, EB, a, b;
  slices(A, d, na, beta, s, EA, a);
  slices(B, d, nb, beta, s, EB, b);
  const long long lim = 1ll << 24;  // FP32 holds every integer of magnitude <= 2^24
  long overflow = 0, bad = 0;
  const int nchunks = (d + chunk - 1) / chunk;
  std::vector<int64_t> D((size_t)s);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) {
      for (int t = 0; t < s; ++t) {
        // one FP32 tensor-memory accumulator per diagonal k + l = t, over each chunk of rows:
        // the MMAs of every pair on the diagonal add into it, one row step at a time
        int64_t total = 0;
        for (int c = 0; c < nchunks; ++c) {
          int64_t part = 0, mag = 0;
          for (int r = c * chunk; r < d && r < (c + 1) * chunk; ++r) {
            for (int k = 0; k <= t; ++k) {
              const int64_t p = (int64_t)a[((size_t)k * na + i) * d + r] *
                                b[((size_t)(t - k) * nb + j) * d + r];
              part += p;
              mag += p < 0 ? -p : p;
            }
          }
          // every partial sum, in any order of addition, is at most the sum of magnitudes
          if (mag > lim) ++overflow;
          total += part;  // the drain of the accumulator, in 64-bit integers
        }
        D[t] = total;
      }
      const double c = cs::oz_combine(D.data(), EA[i], EB[j], beta, s);
      const double want = C[(size_t)i * nb + j];
      uint64_t x, y;
      std::memcpy(&x, &c, 8);
      std::memcpy(&y, &want, 8);
      if (x != y) {
        if (bad < 10) std::printf("C[%d][%d] = %.17g, oracle %.17g\n", i, j, c, want);
        ++bad;
      }
    }
  std::printf("%d x %d over %d rows in chunks of %d (beta %d, %d slices): %ld mismatches, %ld "
              "chunk sums whose magnitudes reach beyond 2^24\n", na, nb, d, chunk, beta, s, bad, overflow);
  return (bad != 0 || overflow != 0) ? 1 : 0;
}
