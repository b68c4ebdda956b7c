// Self-consistent field pieces (include/cs_scf.h): electron density (Sec. 2.1 eq.
// density_expression, Sec. 2.2.5), Hartree potential (Sec. 2.3.1), LDA (Slater exchange +
// Perdew-Zunger correlation), W-weighted grid integrals, Fermi-Dirac occupations by Brent's
// method and Anderson mixing (Sec. 3.4.1), and the SCF step that strings them around the
// ChFSI eigensolver. FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cs_scf.h"
#include "cs_internal.h"
#include "hx_kernels.cuh"

using namespace cs;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kDotBlocks = 608;  // 4 x 152 SMs: fixed partition -> fixed reduction order
constexpr int kDotThreads = 256;

cs_status sfail(cs_ctx* c, cs_status st, const std::string& m) {
  if (c) c->err = m;
  return st;
}

#define SCF_CUDA(c, expr)                                                                 \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return sfail(c, CS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

cs_status ready(cs_ctx* c) {
  if (!c) return CS_ERR_ARG;
  if (!c->has_device) return sfail(c, CS_ERR_STATE, "context has no device");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return sfail(c, CS_ERR_CUDA, cudaGetErrorString(e));
  return CS_OK;
}

long long n_grid(const cs_ctx* c) {
  return (long long)c->host.n_r * c->host.n_theta * c->host.n_phi;
}

// ------------------------------------------------------------------ workspace layout
struct ScfLayout {
  size_t trans;    // cs_inverse_transform / cs_forward_transform workspace
  size_t fgrid;    // CS_DENSITY_CHUNK grid functions
  size_t coef;     // d doubles (Hartree coefficients)
  size_t alm;      // L^2 doubles (harmonic-term amplitudes)
  size_t G1;       // N_r L^2 doubles (Hartree radial synthesis)
  size_t partial;  // kDotBlocks x CS_GRID_INTEGRALS_MAX doubles
  size_t total;
};

ScfLayout scf_layout(const cs_ctx* c) {
  ScfLayout o{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (bytes + 255) & ~size_t(255);
    return at;
  };
  size_t tw = 0;
  cs_workspace_bytes(c, CS_DENSITY_CHUNK, CS_FP64, &tw);
  const HostTables& H = c->host;
  const size_t L2 = (size_t)H.L * H.L;
  o.trans = take(tw);
  o.fgrid = take((size_t)n_grid(c) * CS_DENSITY_CHUNK * 8);
  o.coef = take((size_t)H.d * 8);
  o.alm = take(L2 * 8);
  o.G1 = take((size_t)H.n_r * L2 * 8);
  o.partial = take((size_t)(kDotBlocks + 1) * CS_GRID_INTEGRALS_MAX * 8);  // partials, results
  o.total = off;
  return o;
}

// ------------------------------------------------------------------ kernels
// rho[g] (+)= 2 sum_{s < nc} occ[s] f[s][g]^2, states in order
__global__ void k_density_acc(const double* __restrict__ f, int nc, long long ng,
                              const double* __restrict__ occ, double* __restrict__ rho,
                              int accumulate) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng;
       g += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < nc; ++s) {
      const double v = f[(size_t)s * ng + g];
      acc = fma(occ[s] * v, v, acc);
    }
    rho[g] = (accumulate ? rho[g] : 0.0) + 2.0 * acc;
  }
}

// Per (l, m): vhat_lmn = 4 pi tau_lmn / k_ln^2 (Dirichlet solution) and the amplitude of the
// harmonic term, alm = 4 pi/(2l+1) sqrt(2/R^3) R sum_n tau_lmn / k_ln, so that the term is
// alm (r/R)^l: the multipole moment q_lm = sum_n tau_lmn sqrt(2/R^3) R^(l+2)/k_ln carried to
// the boundary, 4 pi/(2l+1) q_lm r^l / R^(2l+1).
// (vhat may alias tau: each element is read before it is written)
__global__ void k_hartree_coef(const double* tau, int L, int N, const double* __restrict__ kln,
                               double R, double* vhat, double* __restrict__ alm) {
  const int lm = blockIdx.x * blockDim.x + threadIdx.x;
  if (lm >= L * L) return;
  int l = (int)sqrt((double)lm);
  while (l * l > lm) --l;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* t = tau + (size_t)lm * N;
  double* v = vhat + (size_t)lm * N;
  const double* k = kln + (size_t)l * N;
  double s = 0.0;
  for (int n = 0; n < N; ++n) {
    const double tn = t[n];
    s += tn / k[n];
    v[n] = 4.0 * kPi * tn / (k[n] * k[n]);
  }
  alm[lm] = 4.0 * kPi / (2 * l + 1) * sqrt(2.0 / (R * R * R)) * R * s;
}

// G[k][lm] = sum_n R_ln(r_k) vhat_lmn + alm (r_k / R)^l  (one state, layout [k][lm][1])
__global__ void k_hartree_radial(const double* __restrict__ vhat, const double* __restrict__ rad,
                                 const double* __restrict__ alm, const double* __restrict__ rr,
                                 int L, int N, int n_r, double* __restrict__ G) {
  const int L2 = L * L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_r * L2) return;
  const int k = i / L2, lm = i - k * L2;
  int l = (int)sqrt((double)lm);
  while (l * l > lm) --l;
  while ((l + 1) * (l + 1) <= lm) ++l;
  const double* Rk = rad + ((size_t)l * n_r + k) * N;
  const double* v = vhat + (size_t)lm * N;
  double acc = 0.0;
  for (int n = 0; n < N; ++n) acc = fma(Rk[n], v[n], acc);
  G[i] = acc + alm[lm] * pow(rr[k], (double)l);
}

// Perdew-Zunger (1981) fit of the Ceperley-Alder correlation energy, unpolarised
constexpr double kPzGamma = -0.1423, kPzBeta1 = 1.0529, kPzBeta2 = 0.3334;
constexpr double kPzA = 0.0311, kPzB = -0.048, kPzC = 0.0020, kPzD = -0.0116;

__global__ void k_lda(const double* __restrict__ rho, long long n, double* __restrict__ exc,
                      double* __restrict__ vxc) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
       g += (long long)gridDim.x * blockDim.x) {
    const double p = rho[g];
    double e = 0.0, v = 0.0;
    if (p > 0.0) {
      const double c3 = cbrt(3.0 * p / kPi);
      const double ex = -0.75 * c3;                 // Slater exchange per electron
      const double rs = cbrt(3.0 / (4.0 * kPi * p));
      double ec, vc;
      if (rs >= 1.0) {
        const double sq = sqrt(rs);
        const double den = 1.0 + kPzBeta1 * sq + kPzBeta2 * rs;
        ec = kPzGamma / den;
        vc = ec + kPzGamma * (kPzBeta1 * sq / 6.0 + kPzBeta2 * rs / 3.0) / (den * den);
      } else {
        const double lr = log(rs);
        ec = kPzA * lr + kPzB + kPzC * rs * lr + kPzD * rs;
        vc = ec - rs / 3.0 * (kPzA / rs + kPzC * (lr + 1.0) + kPzD);
      }
      e = ex + ec;
      v = 4.0 / 3.0 * ex + vc;
    }
    if (exc) exc[g] = e;
    if (vxc) vxc[g] = v;
  }
}

struct DotArgs {
  const double* f[CS_GRID_INTEGRALS_MAX];
  const double* g[CS_GRID_INTEGRALS_MAX];
  int n;
};

// partial[i][block] = sum over the block's grid-stride points of W_g f_i g_i
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(DotArgs a, const double* __restrict__ wkj,
                                                             int n_phi, long long ng,
                                                             double* __restrict__ partial) {
  __shared__ double red[CS_GRID_INTEGRALS_MAX][kDotThreads / 32];
  double acc[CS_GRID_INTEGRALS_MAX];
#pragma unroll
  for (int i = 0; i < CS_GRID_INTEGRALS_MAX; ++i) acc[i] = 0.0;
  for (long long g = blockIdx.x * (long long)kDotThreads + threadIdx.x; g < ng;
       g += (long long)gridDim.x * kDotThreads) {
    const double w = wkj[g / n_phi];
#pragma unroll
    for (int i = 0; i < CS_GRID_INTEGRALS_MAX; ++i)
      if (i < a.n) acc[i] = fma(w * a.f[i][g], a.g[i] ? a.g[i][g] : 1.0, acc[i]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < CS_GRID_INTEGRALS_MAX; ++i) {
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[i][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < a.n) {
    double s = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) s += red[threadIdx.x][w];
    partial[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void k_dot_reduce(const double* __restrict__ partial, int n, int nb,
                             double* __restrict__ out) {
  const int i = threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[(size_t)i * nb + b];
  out[i] = s;
}

// out[g] = a[g] + b[g] + c[g]
__global__ void k_sum3(const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ c, long long n, double* __restrict__ out) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
       g += (long long)gridDim.x * blockDim.x)
    out[g] = a[g] + b[g] + c[g];
}

// Anderson: V[:, j] = sqrt(W) (F_n - F_{n-j-1}) for j < m, V[:, m] = sqrt(W) F_n
__global__ void k_mix_vectors(const double* const* __restrict__ Fh, int m, long long ng,
                              const double* __restrict__ wkj, int n_phi, double* __restrict__ V) {
  const double* Fn = Fh[0];
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng;
       g += (long long)gridDim.x * blockDim.x) {
    const double sw = sqrt(wkj[g / n_phi]);
    const double fn = Fn[g];
    for (int j = 0; j < m; ++j) V[(size_t)j * ng + g] = sw * (fn - Fh[j + 1][g]);
    V[(size_t)m * ng + g] = sw * fn;
  }
}

// x_next = x_n - sum_j th_j (x_n - x_{n-j}) + beta (F_n - sum_j th_j (F_n - F_{n-j}))
__global__ void k_mix_update(const double* const* __restrict__ xh, const double* const* __restrict__ Fh,
                             const double* __restrict__ th, int m, double beta, long long ng,
                             double* __restrict__ out) {
  const double* xn = xh[0];
  const double* Fn = Fh[0];
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng;
       g += (long long)gridDim.x * blockDim.x) {
    double x = xn[g], F = Fn[g];
    double dx = 0.0, dF = 0.0;
    for (int j = 0; j < m; ++j) {
      dx = fma(th[j], xn[g] - xh[j + 1][g], dx);
      dF = fma(th[j], Fn[g] - Fh[j + 1][g], dF);
    }
    out[g] = (x - dx) + beta * (F - dF);
  }
}

// F = x_out - x_in, and a copy of x_in
__global__ void k_mix_residual(const double* __restrict__ xin, const double* __restrict__ xout,
                               long long ng, double* __restrict__ xs, double* __restrict__ Fs) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng;
       g += (long long)gridDim.x * blockDim.x) {
    const double a = xin[g];
    xs[g] = a;
    Fs[g] = xout[g] - a;
  }
}

unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)std::max<long long>(1, std::min<long long>(b, 152LL * 16));
}

// ------------------------------------------------------------------ host helpers
// Solves A x = b (n x n, row-major copy) by Gaussian elimination with partial pivoting.
bool solve_dense(std::vector<double> A, std::vector<double> b, int n, std::vector<double>& x) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)p * n + c])) p = r;
    if (!(std::fabs(A[(size_t)p * n + c]) > 0.0)) return false;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)p * n + k], A[(size_t)c * n + k]);
      std::swap(b[p], b[c]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
      b[r] -= f * b[c];
    }
  }
  x.assign(n, 0.0);
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[(size_t)r * n + k] * x[k];
    x[r] = s / A[(size_t)r * n + r];
  }
  return true;
}

// softplus(x) = ln(1 + e^x), overflow-free
double softplus(double x) { return std::log1p(std::exp(-std::fabs(x))) + std::max(x, 0.0); }

// Brent's method (Brent 1973, "Algorithms for Minimization without Derivatives", ch. 4):
// root of f on [a, b] with f(a) f(b) <= 0, combining bisection, the secant step and inverse
// quadratic interpolation; tolerance 2 eps |b| + tol.
template <typename Fn>
bool brent_root(Fn f, double a, double b, double tol, double& root) {
  double fa = f(a), fb = f(b);
  if (fa == 0.0) { root = a; return true; }
  if (fb == 0.0) { root = b; return true; }
  if ((fa > 0) == (fb > 0)) return false;
  double c = a, fc = fa, d = b - a, e = d;
  for (int it = 0; it < 500; ++it) {
    if ((fb > 0) == (fc > 0)) {  // keep the root between b and c
      c = a;
      fc = fa;
      d = e = b - a;
    }
    if (std::fabs(fc) < std::fabs(fb)) {  // b is the best estimate
      a = b; b = c; c = a;
      fa = fb; fb = fc; fc = fa;
    }
    const double tol1 = 2.0 * 2.220446049250313e-16 * std::fabs(b) + 0.5 * tol;
    const double xm = 0.5 * (c - b);
    if (std::fabs(xm) <= tol1 || fb == 0.0) {
      root = b;
      return true;
    }
    if (std::fabs(e) >= tol1 && std::fabs(fa) > std::fabs(fb)) {
      double p, q, r;
      const double s = fb / fa;
      if (a == c) {  // secant
        p = 2.0 * xm * s;
        q = 1.0 - s;
      } else {       // inverse quadratic interpolation
        q = fa / fc;
        r = fb / fc;
        p = s * (2.0 * xm * q * (q - r) - (b - a) * (r - 1.0));
        q = (q - 1.0) * (r - 1.0) * (s - 1.0);
      }
      if (p > 0) q = -q;
      p = std::fabs(p);
      const double m1 = 3.0 * xm * q - std::fabs(tol1 * q), m2 = std::fabs(e * q);
      if (2.0 * p < std::min(m1, m2)) {  // accept the interpolation
        e = d;
        d = p / q;
      } else {                           // bisect
        d = xm;
        e = d;
      }
    } else {
      d = xm;
      e = d;
    }
    a = b;
    fa = fb;
    b += (std::fabs(d) > tol1) ? d : (xm > 0 ? tol1 : -tol1);
    fb = f(b);
  }
  root = b;
  return false;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

cs_status cs_scf_workspace_bytes(const cs_ctx* c, size_t* bytes) {
  if (!c || !bytes) return CS_ERR_ARG;
  *bytes = scf_layout(c).total;
  return CS_OK;
}

cs_status cs_density(cs_ctx* c, int n_s, const double* X, long long ld, const double* occ,
                     double* rho, void* work, cs_stream stream) {
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (n_s < 1 || !X || ld < c->host.d || !occ || !rho || !work)
    return sfail(c, CS_ERR_ARG, "cs_density: bad arguments");
  const ScfLayout lay = scf_layout(c);
  char* w = (char*)work;
  double* f = reinterpret_cast<double*>(w + lay.fgrid);
  const long long ng = n_grid(c);
  cudaStream_t st = (cudaStream_t)stream;
  for (int s0 = 0; s0 < n_s; s0 += CS_DENSITY_CHUNK) {
    const int nc = std::min(CS_DENSITY_CHUNK, n_s - s0);
    cs_status r = cs_inverse_transform(c, nc, X + (size_t)s0 * ld, ld, f, w + lay.trans, stream);
    if (r != CS_OK) return r;
    k_density_acc<<<grid_for(ng), 256, 0, st>>>(f, nc, ng, occ + s0, rho, s0 > 0 ? 1 : 0);
    SCF_CUDA(c, cudaGetLastError());
    c->launches += 1;
  }
  return CS_OK;
}

cs_status cs_hartree(cs_ctx* c, const double* rho, double* vh, void* work, cs_stream stream) {
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (!rho || !vh || !work || rho == vh) return sfail(c, CS_ERR_ARG, "cs_hartree: bad arguments");
  const HostTables& H = c->host;
  const ScfLayout lay = scf_layout(c);
  char* w = (char*)work;
  double* coef = reinterpret_cast<double*>(w + lay.coef);
  double* alm = reinterpret_cast<double*>(w + lay.alm);
  double* G1 = reinterpret_cast<double*>(w + lay.G1);
  cudaStream_t st = (cudaStream_t)stream;
  // tau = B^T diag(W) rho
  cs_status r = cs_forward_transform(c, 1, rho, coef, H.d, w + lay.trans, stream);
  if (r != CS_OK) return r;
  const int L2 = H.L * H.L;
  const double* kln = c->hartree_tab;
  const double* rr = c->hartree_tab + (size_t)H.L * H.N;
  k_hartree_coef<<<(L2 + 127) / 128, 128, 0, st>>>(coef, H.L, H.N, kln, H.R, coef, alm);
  SCF_CUDA(c, cudaGetLastError());
  k_hartree_radial<<<(H.n_r * L2 + 255) / 256, 256, 0, st>>>(coef, c->d64.rad, alm, rr, H.L,
                                                               H.N, H.n_r, G1);
  SCF_CUDA(c, cudaGetLastError());
  AngArgs<double> a{H.L, H.n_r, H.n_theta, H.n_phi, c->Q4, 1, c->d64.theta, c->d64.trig,
                    c->d64.wv, c->d64.wkj};
  SCF_CUDA(c, launch_angular<double>(a, ANG_SYNTH, G1, vh, nullptr, st));
  c->launches += 3;
  return CS_OK;
}

cs_status cs_lda_xc(cs_ctx* c, const double* rho, double* exc, double* vxc, cs_stream stream) {
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (!rho || (!exc && !vxc)) return sfail(c, CS_ERR_ARG, "cs_lda_xc: bad arguments");
  const long long ng = n_grid(c);
  k_lda<<<grid_for(ng), 256, 0, (cudaStream_t)stream>>>(rho, ng, exc, vxc);
  SCF_CUDA(c, cudaGetLastError());
  c->launches += 1;
  return CS_OK;
}

cs_status cs_grid_integrals(cs_ctx* c, int n, const double* const* f, const double* const* g,
                            double* out, void* work, cs_stream stream) {
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (n < 1 || n > CS_GRID_INTEGRALS_MAX || !f || !out || !work)
    return sfail(c, CS_ERR_ARG, "cs_grid_integrals: bad arguments");
  DotArgs a{};
  a.n = n;
  for (int i = 0; i < n; ++i) {
    if (!f[i]) return sfail(c, CS_ERR_ARG, "cs_grid_integrals: NULL f");
    a.f[i] = f[i];
    a.g[i] = g ? g[i] : nullptr;
  }
  const ScfLayout lay = scf_layout(c);
  double* partial = reinterpret_cast<double*>((char*)work + lay.partial);
  double* res = partial + (size_t)kDotBlocks * CS_GRID_INTEGRALS_MAX;
  cudaStream_t st = (cudaStream_t)stream;
  k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(a, c->d64.wkj, c->host.n_phi, n_grid(c),
                                                    partial);
  SCF_CUDA(c, cudaGetLastError());
  k_dot_reduce<<<1, 32, 0, st>>>(partial, n, kDotBlocks, res);
  SCF_CUDA(c, cudaGetLastError());
  c->launches += 2;
  SCF_CUDA(c, cudaMemcpyAsync(out, res, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  SCF_CUDA(c, cudaStreamSynchronize(st));
  return CS_OK;
}

cs_status cs_fermi_occupations(int n, const double* lambda, double n_electrons, double kT,
                               double* occ, double* mu, double* entropy) {
  if (n < 1 || !lambda || !occ || !(kT > 0.0)) return CS_ERR_ARG;
  const double target = 0.5 * n_electrons;
  if (!(target > 0.0 && target < n)) return CS_ERR_ARG;
  double lo = lambda[0], hi = lambda[0];
  for (int i = 1; i < n; ++i) {
    lo = std::min(lo, lambda[i]);
    hi = std::max(hi, lambda[i]);
  }
  auto count = [&](double m) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
      const double x = (lambda[i] - m) / kT;
      s += (x >= 0) ? std::exp(-x) / (1.0 + std::exp(-x)) : 1.0 / (1.0 + std::exp(x));
    }
    return s - target;
  };
  double m = 0.0;
  if (!brent_root(count, lo - 60.0 * kT - 1.0, hi + 60.0 * kT + 1.0, 1e-15, m))
    return CS_ERR_NOT_CONVERGED;
  double S = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = (lambda[i] - m) / kT;
    const double f = (x >= 0) ? std::exp(-x) / (1.0 + std::exp(-x)) : 1.0 / (1.0 + std::exp(x));
    occ[i] = f;
    // f ln f + (1-f) ln(1-f) = -f softplus(x) - (1-f) softplus(-x)
    S += f * softplus(x) + (1.0 - f) * softplus(-x);
  }
  if (mu) *mu = m;
  if (entropy) *entropy = 2.0 * S;
  return CS_OK;
}

}  // extern "C"

// ====================================================================== mixer
struct cs_mixer {
  cs_ctx* ctx = nullptr;
  double beta = 0.3;
  int history = 0;
  int count = 0;    // iterates stored (<= history + 1)
  int head = 0;     // slot of the newest iterate
  long long ng = 0;
  double* xs = nullptr;     // [history + 1][ng]
  double* Fs = nullptr;     // [history + 1][ng]
  double* V = nullptr;      // [(history + 1)][ng] weighted differences
  double* gram = nullptr;   // (history + 1)^2
  double* partial = nullptr;
  double* th = nullptr;     // history
  const double** ptrs = nullptr;  // device: 2 (history + 1) pointers
  std::vector<double> hgram;
};

extern "C" {

cs_status cs_mixer_create(cs_ctx* c, double beta, int history, cs_mixer** out) {
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (!out || !(beta > 0.0 && beta <= 1.0) || history < 0 || history > CS_MIXER_MAX_HISTORY)
    return sfail(c, CS_ERR_ARG, "cs_mixer_create: need 0 < beta <= 1, 0 <= history <= 64");
  cs_mixer* m = new cs_mixer;
  m->ctx = c;
  m->beta = beta;
  m->history = history;
  m->ng = n_grid(c);
  const int slots = history + 1;
  const size_t pe = gram_partial_elems(m->ng, slots, slots);
  bool ok = cudaMalloc((void**)&m->xs, (size_t)slots * m->ng * 8) == cudaSuccess &&
            cudaMalloc((void**)&m->Fs, (size_t)slots * m->ng * 8) == cudaSuccess &&
            cudaMalloc((void**)&m->V, (size_t)slots * m->ng * 8) == cudaSuccess &&
            cudaMalloc((void**)&m->gram, (size_t)slots * slots * 8) == cudaSuccess &&
            cudaMalloc((void**)&m->partial, std::max<size_t>(pe, 1) * 8) == cudaSuccess &&
            cudaMalloc((void**)&m->th, (size_t)slots * 8) == cudaSuccess &&
            cudaMalloc((void**)&m->ptrs, 2 * (size_t)slots * sizeof(double*)) == cudaSuccess;
  if (!ok) {
    cs_mixer_free(m);
    return sfail(c, CS_ERR_ALLOC, "cs_mixer_create: cudaMalloc failed");
  }
  *out = m;
  return CS_OK;
}

cs_status cs_mixer_reset(cs_mixer* m) {
  if (!m) return CS_ERR_ARG;
  m->count = 0;
  m->head = 0;
  return CS_OK;
}

cs_status cs_mixer_mix(cs_mixer* m, const double* x_in, const double* x_out, double* x_next,
                       cs_stream stream) {
  if (!m) return CS_ERR_ARG;
  cs_ctx* c = m->ctx;
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (!x_in || !x_out || !x_next) return sfail(c, CS_ERR_ARG, "cs_mixer_mix: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int slots = m->history + 1;
  const long long ng = m->ng;
  // store the newest iterate and residual
  m->head = (m->count == 0) ? 0 : (m->head + 1) % slots;
  m->count = std::min(m->count + 1, slots);
  double* xn = m->xs + (size_t)m->head * ng;
  double* Fn = m->Fs + (size_t)m->head * ng;
  k_mix_residual<<<grid_for(ng), 256, 0, st>>>(x_in, x_out, ng, xn, Fn);
  SCF_CUDA(c, cudaGetLastError());
  const int mm = m->count - 1;  // previous iterates in use
  // pointer tables: [0] newest, [j] the j-th previous
  std::vector<const double*> hp(2 * (size_t)slots, nullptr);
  for (int j = 0; j <= mm; ++j) {
    const int slot = (m->head - j + slots) % slots;
    hp[j] = m->xs + (size_t)slot * ng;
    hp[slots + j] = m->Fs + (size_t)slot * ng;
  }
  SCF_CUDA(c, cudaMemcpyAsync(m->ptrs, hp.data(), hp.size() * sizeof(double*),
                              cudaMemcpyHostToDevice, st));
  std::vector<double> theta(std::max(mm, 1), 0.0);
  if (mm > 0) {
    k_mix_vectors<<<grid_for(ng), 256, 0, st>>>(m->ptrs + slots, mm, ng, c->d64.wkj,
                                                c->host.n_phi, m->V);
    SCF_CUDA(c, cudaGetLastError());
    const int nv = mm + 1;
    SCF_CUDA(c, launch_gram<double>(m->V, ng, m->V, ng, ng, nv, nv, m->gram, nv, m->partial, st));
    m->hgram.resize((size_t)nv * nv);
    SCF_CUDA(c, cudaMemcpyAsync(m->hgram.data(), m->gram, (size_t)nv * nv * 8,
                                cudaMemcpyDeviceToHost, st));
    SCF_CUDA(c, cudaStreamSynchronize(st));
    std::vector<double> A((size_t)mm * mm), b(mm);
    for (int j = 0; j < mm; ++j) {
      for (int k = 0; k < mm; ++k) A[(size_t)j * mm + k] = m->hgram[(size_t)k * nv + j];
      b[j] = m->hgram[(size_t)mm * nv + j];
    }
    std::vector<double> x;
    if (!solve_dense(A, b, mm, x)) return sfail(c, CS_ERR_NUMERIC, "cs_mixer_mix: singular Gram");
    for (int j = 0; j < mm; ++j) theta[j] = x[j];
    SCF_CUDA(c, cudaMemcpyAsync(m->th, theta.data(), mm * sizeof(double),
                                cudaMemcpyHostToDevice, st));
    c->launches += 3;
  }
  k_mix_update<<<grid_for(ng), 256, 0, st>>>(m->ptrs, m->ptrs + slots, m->th, mm, m->beta, ng,
                                             x_next);
  SCF_CUDA(c, cudaGetLastError());
  c->launches += 2;
  // the host vectors hold the pointer table and theta until the copies have run
  SCF_CUDA(c, cudaStreamSynchronize(st));
  return CS_OK;
}

cs_status cs_mixer_free(cs_mixer* m) {
  if (!m) return CS_OK;
  if (m->ctx && m->ctx->has_device) cudaSetDevice(m->ctx->device);
  for (void* p : {(void*)m->xs, (void*)m->Fs, (void*)m->V, (void*)m->gram, (void*)m->partial,
                  (void*)m->th, (void*)m->ptrs})
    if (p) cudaFree(p);
  delete m;
  return CS_OK;
}

}  // extern "C"

// ====================================================================== SCF loop
struct cs_scf {
  cs_ctx* ctx = nullptr;
  cs_scf_params p{};
  long long ng = 0;
  double* v_ext = nullptr;
  double* v_in = nullptr;
  double* v_out = nullptr;
  double* rho = nullptr;
  double* vh = nullptr;
  double* exc = nullptr;
  double* vxc = nullptr;
  double* occ_dev = nullptr;
  double* v0 = nullptr;
  cs_mixer* mixer = nullptr;
  int iteration = 0;
  double e_prev = 0.0;
  std::vector<double> theta_h, occ_h, resid_h;
};

extern "C" {

cs_status cs_scf_create(cs_ctx* c, const cs_scf_params* p, const double* v_ext,
                        const double* rho0, const double* v0, cs_scf** out) {
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (!p || !v_ext || !rho0 || !v0 || !out) return sfail(c, CS_ERR_ARG, "cs_scf_create: NULL argument");
  if (p->n_s < 1 || p->n_want < 1 || p->n_want > p->n_s || p->degree < 1 || !(p->kT > 0) ||
      !(0.5 * p->n_electrons > 0 && 0.5 * p->n_electrons < p->n_s) || p->lanczos_k < 1 ||
      p->lanczos_k > 64 || p->first_max_iter < 1 || p->first_solver < 0 || p->first_solver > 1)
    return sfail(c, CS_ERR_ARG, "cs_scf_create: bad parameters");
  cs_scf* S = new cs_scf;
  S->ctx = c;
  S->p = *p;
  S->ng = n_grid(c);
  const size_t gb = (size_t)S->ng * 8;
  bool ok = true;
  for (double** q : {&S->v_ext, &S->v_in, &S->v_out, &S->rho, &S->vh, &S->exc, &S->vxc})
    ok = ok && cudaMalloc((void**)q, gb) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&S->occ_dev, (size_t)p->n_s * 8) == cudaSuccess &&
       cudaMalloc((void**)&S->v0, (size_t)c->host.d * 8) == cudaSuccess;
  if (!ok) {
    cs_scf_free(S);
    return sfail(c, CS_ERR_ALLOC, "cs_scf_create: cudaMalloc failed");
  }
  if ((s = cs_mixer_create(c, p->beta, p->history, &S->mixer)) != CS_OK) {
    cs_scf_free(S);
    return s;
  }
  // the starting density is kept in `rho` until the first step builds v_in from it
  if (cudaMemcpy(S->v_ext, v_ext, gb, cudaMemcpyDeviceToDevice) != cudaSuccess ||
      cudaMemcpy(S->rho, rho0, gb, cudaMemcpyDeviceToDevice) != cudaSuccess ||
      cudaMemcpy(S->v0, v0, (size_t)c->host.d * 8, cudaMemcpyDeviceToDevice) != cudaSuccess) {
    cs_scf_free(S);
    return sfail(c, CS_ERR_CUDA, "cs_scf_create: copies failed");
  }
  S->theta_h.assign(p->n_s, 0.0);
  S->occ_h.assign(p->n_s, 0.0);
  S->resid_h.assign(p->n_s, 0.0);
  *out = S;
  return CS_OK;
}

cs_status cs_scf_work_bytes(const cs_scf* S, size_t* bytes) {
  if (!S || !bytes) return CS_ERR_ARG;
  size_t a = 0, b = 0;
  cs_workspace_bytes(S->ctx, S->p.n_s, S->p.filter_prec, &a);
  cs_workspace_bytes(S->ctx, S->p.n_s, CS_FP64, &b);
  *bytes = std::max(std::max(a, b), scf_layout(S->ctx).total);
  if (S->p.first_solver == 1) {
    size_t l = 0;
    cs_lobpcg_workspace_bytes(S->ctx, S->p.n_s, &l);
    *bytes = std::max(*bytes, l);
  }
  return CS_OK;
}

cs_status cs_scf_step(cs_scf* S, double* X, long long ld, double* theta, double* resid,
                      void* work, cs_stream stream, cs_scf_report* rep) {
  if (!S) return CS_ERR_ARG;
  cs_ctx* c = S->ctx;
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  if (!X || ld < c->host.d || !theta || !resid || !work || !rep)
    return sfail(c, CS_ERR_ARG, "cs_scf_step: bad arguments");
  const cs_scf_params& p = S->p;
  cudaStream_t st = (cudaStream_t)stream;
  const long long ng = S->ng;
  if (S->iteration == 0) {  // v_in = v_ext + V_H[rho0] + v_xc[rho0]
    if ((s = cs_hartree(c, S->rho, S->vh, work, stream)) != CS_OK) return s;
    if ((s = cs_lda_xc(c, S->rho, nullptr, S->vxc, stream)) != CS_OK) return s;
    k_sum3<<<grid_for(ng), 256, 0, st>>>(S->v_ext, S->vh, S->vxc, ng, S->v_in);
    SCF_CUDA(c, cudaGetLastError());
    c->launches += 1;
  }
  if ((s = cs_set_potential(c, S->v_in, stream)) != CS_OK) return s;
  int iters = 1;
  if (S->iteration == 0) {
    if (p.first_solver == 1)
      s = cs_lobpcg(c, p.n_s, p.n_want, X, ld, p.first_tol, p.first_max_iter, 1, theta, resid,
                    &iters, nullptr, work, stream);
    else
      s = cs_chfsi(c, p.n_s, p.n_want, X, ld, p.degree, p.first_tol, p.first_max_iter,
                   p.filter_prec, S->v0, theta, resid, &iters, work, stream);
    if (s != CS_OK && s != CS_ERR_NOT_CONVERGED) return s;
  } else {
    double b = 0.0, tmin = 0.0;
    if ((s = cs_lanczos_bound(c, p.lanczos_k, S->v0, &b, &tmin, work, stream)) != CS_OK) return s;
    const double a0 = S->theta_h[0], a = S->theta_h[p.n_s - 1];
    if (!(b > a)) b = a + std::max(0.1 * (a - a0), 1e-3);
    if ((s = cs_chfsi_step(c, p.n_s, X, ld, p.degree, a, b, std::min(a0, a - 1e-9 * std::fabs(a) - 1e-12),
                           p.filter_prec, theta, resid, work, stream)) != CS_OK)
      return s;
  }
  SCF_CUDA(c, cudaMemcpyAsync(S->theta_h.data(), theta, p.n_s * 8, cudaMemcpyDeviceToHost, st));
  SCF_CUDA(c, cudaMemcpyAsync(S->resid_h.data(), resid, p.n_s * 8, cudaMemcpyDeviceToHost, st));
  SCF_CUDA(c, cudaStreamSynchronize(st));
  double mu = 0.0, ent = 0.0;
  if ((s = cs_fermi_occupations(p.n_s, S->theta_h.data(), p.n_electrons, p.kT, S->occ_h.data(),
                                &mu, &ent)) != CS_OK)
    return sfail(c, s, "cs_scf_step: Fermi level not found");
  SCF_CUDA(c, cudaMemcpyAsync(S->occ_dev, S->occ_h.data(), p.n_s * 8, cudaMemcpyHostToDevice, st));
  if ((s = cs_density(c, p.n_s, X, ld, S->occ_dev, S->rho, work, stream)) != CS_OK) return s;
  if ((s = cs_hartree(c, S->rho, S->vh, work, stream)) != CS_OK) return s;
  if ((s = cs_lda_xc(c, S->rho, S->exc, S->vxc, stream)) != CS_OK) return s;
  const double* fs[4] = {S->rho, S->rho, S->rho, S->rho};
  const double* gs[4] = {S->v_in, S->v_ext, S->vh, S->exc};
  double I[4];
  if ((s = cs_grid_integrals(c, 4, fs, gs, I, work, stream)) != CS_OK) return s;
  double band = 0.0;
  for (int i = 0; i < p.n_s; ++i) band += 2.0 * S->occ_h[i] * S->theta_h[i];
  const double E = band - (I[0] - I[1]) + 0.5 * I[2] + I[3] - p.kT * ent + p.e_ion;
  // v_out = v_ext + V_H + v_xc, then v_in <- mix(v_in, v_out)
  k_sum3<<<grid_for(ng), 256, 0, st>>>(S->v_ext, S->vh, S->vxc, ng, S->v_out);
  SCF_CUDA(c, cudaGetLastError());
  c->launches += 1;
  if ((s = cs_mixer_mix(S->mixer, S->v_in, S->v_out, S->v_in, stream)) != CS_OK) return s;
  double mr = 0.0;
  for (double r : S->resid_h) mr = std::max(mr, r);
  S->iteration += 1;
  rep->iteration = S->iteration;
  rep->chfsi_iterations = iters;
  rep->energy = E;
  rep->dE = (S->iteration == 1) ? 0.0 : E - S->e_prev;
  rep->mu = mu;
  rep->entropy = ent;
  rep->band = band;
  rep->e_hartree = 0.5 * I[2];
  rep->e_xc = I[3];
  rep->max_resid = mr;
  S->e_prev = E;
  return CS_OK;
}

cs_status cs_scf_grid(const cs_scf* S, int which, double* out, cs_stream stream) {
  if (!S || !out) return CS_ERR_ARG;
  const double* src = nullptr;
  switch (which) {
    case 0: src = S->v_in; break;
    case 1: src = S->rho; break;
    case 2: src = S->vh; break;
    case 3: src = S->exc; break;
    case 4: src = S->v_ext; break;
    default: return sfail(S->ctx, CS_ERR_ARG, "cs_scf_grid: unknown grid function");
  }
  cs_ctx* c = S->ctx;
  cs_status s = ready(c);
  if (s != CS_OK) return s;
  SCF_CUDA(c, cudaMemcpyAsync(out, src, (size_t)S->ng * 8, cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return CS_OK;
}

cs_status cs_scf_occupations(const cs_scf* S, double* occ) {
  if (!S || !occ) return CS_ERR_ARG;
  std::memcpy(occ, S->occ_h.data(), S->occ_h.size() * 8);
  return CS_OK;
}

cs_status cs_scf_free(cs_scf* S) {
  if (!S) return CS_OK;
  if (S->ctx && S->ctx->has_device) {
    cudaSetDevice(S->ctx->device);
    cudaDeviceSynchronize();
  }
  for (double* q : {S->v_ext, S->v_in, S->v_out, S->rho, S->vh, S->exc, S->vxc, S->occ_dev, S->v0})
    if (q) cudaFree(q);
  cs_mixer_free(S->mixer);
  delete S;
  return CS_OK;
}

}  // extern "C"
