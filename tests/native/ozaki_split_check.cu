// Host check of the integer slices (ozaki_split.cuh) against digits written by the FP64 oracle.
// Input file: int32 d, n, beta, s; then X (d x n FP64, column-major); then the oracle's column
// exponents (n int64) and digits (s x d x n int64, digit-major then row-major over (r, j)).
// Exit status 0 when every exponent and digit agrees.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../paper_1404_3773_gb300/csrc/ozaki_split.cuh"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[4];
  if (std::fread(hdr, 4, 4, f) != 4) return 2;
  const int d = hdr[0], n = hdr[1], beta = hdr[2], s = hdr[3];
  std::vector<double> X((size_t)d * n);
  std::vector<int64_t> E(n), A((size_t)s * d * n);
  if (std::fread(X.data(), 8, X.size(), f) != X.size()) return 2;
  if (std::fread(E.data(), 8, E.size(), f) != E.size()) return 2;
  if (std::fread(A.data(), 8, A.size(), f) != A.size()) return 2;
  std::fclose(f);
  long bad = 0;
  std::vector<int> a(s);
  for (int j = 0; j < n; ++j) {
    double m = 0.0;
    for (int r = 0; r < d; ++r) m = std::fmax(m, std::fabs(X[(size_t)j * d + r]));
    const int Ej = cs::oz_exponent(m);
    if (Ej != (int)E[j]) {
      if (bad < 10) std::printf("column %d: exponent %d, oracle %lld\n", j, Ej, (long long)E[j]);
      ++bad;
      continue;
    }
    for (int r = 0; r < d; ++r) {
      cs::oz_slices(X[(size_t)j * d + r], Ej, beta, s, a.data());
      for (int k = 0; k < s; ++k) {
        const int64_t want = A[((size_t)k * d + r) * n + j];
        if (a[k] != want) {
          if (bad < 10)
            std::printf("x = %.17g (r %d, col %d): digit %d is %d, oracle %lld\n",
                        X[(size_t)j * d + r], r, j, k, a[k], (long long)want);
          ++bad;
        }
      }
    }
  }
  std::printf("%d x %d values, beta %d, %d slices: %ld mismatches\n", d, n, beta, s, bad);
  return bad != 0;
}
