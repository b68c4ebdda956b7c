// Host-side set-up of the basis tables (double precision, once per basis).
//
// Sec. 2.2.1: R_ln(r) = J_{l+1/2}(b r/R) sqrt(2/r) / (R J_{l+3/2}(b)), b = b^n_{l+1/2}, which
// with j_l(x) = sqrt(pi/(2x)) J_{l+1/2}(x) is sqrt(2/R^3) j_l(b r/R) / j_{l+1}(b).
// Sec. 3.4.2: the zeros b^n_{l+1/2} are found with Halley's method; the Gauss rules
// (Sec. 2.2.2) are built here by Newton iteration on the orthogonal polynomials.
// eq. spherical_harmonics_1: c_lm P_l^m(cos theta), no Condon-Shortley phase.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "cs_internal.h"

namespace cs {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

// j_l(x) for x >= 0. x > l: forward recurrence from j_0, j_1 (the minimal solution
// grows in that direction while n < x). Otherwise: backward recurrence from order
// l + 40 on an arbitrary seed, normalised with the sum rule sum_n (2n+1) j_n(x)^2 = 1
// (accumulated with rescaling so that no value overflows).
double sph_j(int l, double x) {
  if (x == 0.0) return l == 0 ? 1.0 : 0.0;
  const double s = std::sin(x), c = std::cos(x);
  if (l == 0) return s / x;
  if (x > l) {
    double a = s / x, b = s / (x * x) - c / x;
    for (int n = 1; n < l; ++n) {
      double nb = (2 * n + 1) / x * b - a;
      a = b;
      b = nb;
    }
    return b;
  }
  const int top = l + 40;
  double up = 0.0, cur = 1e-280;  // orders top+1, top
  long double sum = (long double)(2 * top + 1) * cur * cur;
  double at_l = 0.0;
  for (int n = top; n >= 1; --n) {
    double lower = (2 * n + 1) / x * cur - up;  // order n-1
    up = cur;
    cur = lower;
    if (n - 1 == l) at_l = cur;
    sum += (long double)(2 * (n - 1) + 1) * (long double)cur * cur;
    if (std::fabs(cur) > 1e150) {  // rescale everything kept so far
      up *= 1e-150;
      cur *= 1e-150;
      at_l *= 1e-150;
      sum *= 1e-300L;
    }
  }
  return (double)((long double)at_l / std::sqrt(sum));
}

// d/dx j_l = j_{l-1} - (l+1)/x j_l ;  j_l'' from the spherical Bessel equation
void sph_j_derivs(int l, double x, double& f, double& f1, double& f2) {
  f = sph_j(l, x);
  f1 = (l == 0) ? -sph_j(1, x) : sph_j(l - 1, x) - (l + 1) / x * f;
  f2 = -2.0 / x * f1 - (1.0 - l * (l + 1) / (x * x)) * f;
}

// zero of j_l inside (lo, hi) where j_l changes sign: Halley steps, bisection fallback
double halley_zero(int l, double lo, double hi) {
  double flo = sph_j(l, lo);
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double f, f1, f2;
    sph_j_derivs(l, x, f, f1, f2);
    if (f == 0.0) return x;
    if ((f > 0) == (flo > 0)) {
      lo = x;
      flo = f;
    } else {
      hi = x;
    }
    double step = 2.0 * f * f1 / (2.0 * f1 * f1 - f * f2);
    double xn = x - step;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) <= 2e-16 * std::fabs(x)) return xn;
    x = xn;
  }
  return x;
}

// Gauss-Legendre on [-1,1], ascending nodes
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    // guess for the i-th largest root, refined by Newton on P_n
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (n == 1) p0 = 1.0;
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;  // roots come out descending
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Jacobi polynomial P_n^{(0,2)} and its derivative at x
void jacobi02(int n, double x, double& p, double& dp) {
  const double a = 0.0, b = 2.0;
  double pm1 = 1.0;
  double pc = (a + 1.0) + (a + b + 2.0) * (x - 1.0) / 2.0;
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double s = 2.0 * k + a + b;
    double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
    double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
    double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
    double pn = (c2 * pc - c3 * pm1) / c1;
    pm1 = pc;
    pc = pn;
  }
  p = pc;
  double s = 2.0 * n + a + b;
  // (2n+a+b)(1-x^2) P_n' = n[(a-b) - (2n+a+b)x] P_n + 2(n+a)(n+b) P_{n-1}
  dp = (n * ((a - b) - s * x) * pc + 2.0 * (n + a) * (n + b) * pm1) / (s * (1.0 - x * x));
}

// Gauss-Jacobi (alpha = 0, beta = 2) on [-1,1], ascending: roots bracketed on a fine
// uniform theta grid (x = cos theta), bisection then Newton polish; weights
// w = 2^3 / ((1 - x^2) P_n'(x)^2).
void gauss_jacobi02(int n, std::vector<double>& x, std::vector<double>& w) {
  x.clear();
  w.clear();
  const int M = 32 * n + 64;
  double th_prev = kPi, p_prev, dpd;
  jacobi02(n, std::cos(th_prev), p_prev, dpd);
  for (int i = M - 1; i >= 0; --i) {
    double th = kPi * i / M;
    double p, dpx;
    jacobi02(n, std::cos(th), p, dpx);
    if ((p > 0) != (p_prev > 0) || p == 0.0) {
      double lo = std::cos(th_prev), hi = std::cos(th), flo = p_prev;
      for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
        double mid = 0.5 * (lo + hi), fm, dm;
        jacobi02(n, mid, fm, dm);
        if ((fm > 0) == (flo > 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      double z = 0.5 * (lo + hi);
      for (int it = 0; it < 3; ++it) {
        double f, df;
        jacobi02(n, z, f, df);
        z -= f / df;
      }
      double f, df;
      jacobi02(n, z, f, df);
      x.push_back(z);
      w.push_back(8.0 / ((1.0 - z * z) * df * df));
    }
    th_prev = th;
    p_prev = p;
  }
}

// normalised Theta_lm(t) = c_lm P_l^m(t) (no Condon-Shortley phase), all 0 <= m <= l <= lmax
void legendre_row(int lmax, double t, std::vector<double>& th /* [(l)(lmax+1)+m] */) {
  const int L = lmax + 1;
  th.assign((size_t)L * L, 0.0);
  const double st = std::sqrt(std::fmax(0.0, 1.0 - t * t));
  double pmm = 1.0 / std::sqrt(4.0 * kPi);
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) pmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * st;
    th[(size_t)m * L + m] = pmm;
    if (m + 1 <= lmax) th[(size_t)(m + 1) * L + m] = std::sqrt(2.0 * m + 3.0) * t * pmm;
    for (int l = m + 2; l <= lmax; ++l) {
      double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) /
                           (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
      th[(size_t)l * L + m] = a * (t * th[(size_t)(l - 1) * L + m] - b * th[(size_t)(l - 2) * L + m]);
    }
  }
}

}  // namespace

std::string build_host_tables(double R, int lmax, int nmax, const cs_quadrature& q,
                              HostTables& T) {
  if (!(R > 0.0)) return "R must be positive";
  if (lmax < 0 || lmax > 400) return "lmax out of range [0, 400]";
  if (nmax < 1 || nmax > 4096) return "nmax out of range [1, 4096]";
  if (q.n_r < 1 || q.n_r > 4096) return "n_r out of range [1, 4096]";
  if (q.n_theta <= lmax || q.n_theta > 4096) return "n_theta must be > lmax (and <= 4096)";
  if (q.n_phi % 2 != 0 || q.n_phi < 2 * lmax + 2 || q.n_phi > 8192)
    return "n_phi must be even and >= 2*lmax+2 (and <= 8192)";
  if (q.radial != CS_RADIAL_GAUSS_LEGENDRE && q.radial != CS_RADIAL_GAUSS_JACOBI_R2)
    return "unknown radial rule";
  T.R = R;
  T.lmax = lmax;
  T.L = lmax + 1;
  T.N = nmax;
  T.d = (long long)T.L * T.L * nmax;
  T.n_r = q.n_r;
  T.n_theta = q.n_theta;
  T.n_phi = q.n_phi;
  T.radial = q.radial;
  const int L = T.L, N = nmax;

  // radial rule on [0, R], weights including r^2
  std::vector<double> x, w;
  if (q.radial == CS_RADIAL_GAUSS_LEGENDRE) {
    gauss_legendre(q.n_r, x, w);
    T.r.resize(q.n_r);
    T.w_r.resize(q.n_r);
    for (int k = 0; k < q.n_r; ++k) {
      T.r[k] = 0.5 * R * (1.0 + x[k]);
      T.w_r[k] = 0.5 * R * w[k] * T.r[k] * T.r[k];
    }
  } else {
    gauss_jacobi02(q.n_r, x, w);
    if ((int)x.size() != q.n_r) return "Gauss-Jacobi root search failed";
    T.r.resize(q.n_r);
    T.w_r.resize(q.n_r);
    for (int k = 0; k < q.n_r; ++k) {
      T.r[k] = 0.5 * R * (1.0 + x[k]);
      T.w_r[k] = 0.125 * R * R * R * w[k];
    }
  }
  gauss_legendre(q.n_theta, T.t, T.w_t);
  T.phi.resize(q.n_phi);
  for (int j = 0; j < q.n_phi; ++j) T.phi[j] = 2.0 * kPi * j / q.n_phi;

  // zeros: z_0n = (n+1) pi; z_{l,n} lies between z_{l-1,n} and z_{l-1,n+1}
  const int cnt = N + L;
  std::vector<double> prev(cnt), cur(cnt);
  for (int n = 0; n < cnt; ++n) prev[n] = kPi * (n + 1);
  T.z.assign((size_t)L * N, 0.0);
  for (int n = 0; n < N; ++n) T.z[n] = prev[n];
  for (int l = 1; l < L; ++l) {
    int c = cnt - l;
    for (int n = 0; n < c; ++n) cur[n] = halley_zero(l, prev[n], prev[n + 1]);
    for (int n = 0; n < N; ++n) T.z[(size_t)l * N + n] = cur[n];
    std::swap(prev, cur);
  }

  // radial table
  T.rad.assign((size_t)L * q.n_r * N, 0.0);
  const double pre = std::sqrt(2.0 / (R * R * R));
  for (int l = 0; l < L; ++l)
    for (int n = 0; n < N; ++n) {
      double zz = T.z[(size_t)l * N + n];
      double nrm = pre / sph_j(l + 1, zz);
      for (int k = 0; k < q.n_r; ++k)
        T.rad[((size_t)l * q.n_r + k) * N + n] = nrm * sph_j(l, zz * T.r[k] / R);
    }

  // theta rows (sqrt2 folded in for m > 0)
  const int rowlen = theta_row_len(L);
  T.theta.assign((size_t)q.n_theta * rowlen, 0.0);
  std::vector<double> th;
  for (int j = 0; j < q.n_theta; ++j) {
    legendre_row(lmax, T.t[j], th);
    for (int m = 0; m < L; ++m)
      for (int l = m; l < L; ++l)
        T.theta[(size_t)j * rowlen + theta_off(L, m) + (l - m)] =
            th[(size_t)l * L + m] * (m > 0 ? std::sqrt(2.0) : 1.0);
  }

  T.half_lambda.assign((size_t)T.d, 0.0);
  for (int l = 0; l < L; ++l)
    for (int m = -l; m <= l; ++m)
      for (int n = 0; n < N; ++n) {
        double k = T.z[(size_t)l * N + n] / R;
        T.half_lambda[(size_t)(l * l + l + m) * N + n] = 0.5 * k * k;
      }
  return std::string();
}

}  // namespace cs
