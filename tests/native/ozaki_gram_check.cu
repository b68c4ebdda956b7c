// Host check of the whole slice-product pipeline of ozaki_split.cuh: split both operands,
// form the exact integer sum of the slice products on each diagonal k + l = t, combine
// (oz_combine: exact sum, one rounding), and compare with the oracle's C = A^T B bit for bit. Input file: int32 d, na, nb, beta, s; A (d x na, FP64,
// column-major); B (d x nb); the oracle's C (na x nb, row-major). Exit status 0 on agreement.
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
  int32_t h[5];
  if (std::fread(h, 4, 5, f) != 5) return 2;
  const int d = h[0], na = h[1], nb = h[2], beta = h[3], s = h[4];
  std::vector<double> A((size_t)d * na), B((size_t)d * nb), C((size_t)na * nb);
  if (std::fread(A.data(), 8, A.size(), f) != A.size()) return 2;
  if (std::fread(B.data(), 8, B.size(), f) != B.size()) return 2;
  if (std::fread(C.data(), 8, C.size(), f) != C.size()) return 2;
  std::fclose(f);
  std::vector<int> EA, EB, a, b;
  slices(A, d, na, beta, s, EA, a);
  slices(B, d, nb, beta, s, EB, b);
  long bad = 0;
  std::vector<int64_t> D((size_t)s);
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) {
      // exact diagonal sums D_t = sum_{k + l = t} a_k^T b_l
      for (int t = 0; t < s; ++t) {
        int64_t acc = 0;
        for (int k = 0; k <= t; ++k) {
          const int* ak = &a[((size_t)k * na + i) * d];
          const int* bl = &b[((size_t)(t - k) * nb + j) * d];
          for (int r = 0; r < d; ++r) acc += (int64_t)ak[r] * bl[r];
        }
        D[t] = acc;
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
  std::printf("%d x %d entries over %d rows, beta %d, %d slices: %ld mismatches\n", na, nb, d,
              beta, s, bad);
  return bad != 0;
}
