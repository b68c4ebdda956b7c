// Learned initial SCF density (include/cs_learned.h): per-atom radial descriptors (host), the
// atom-centred Gaussian density expansion on the grid and its weighted least-squares fit, and a
// tanh multilayer perceptron with mean-squared-error gradients and Adam, all in FP32 apart
// from the grid work (FP64).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cs_learned.h"
#include "cs_internal.h"
#include "hx_kernels.cuh"

using namespace cs;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxBasis = 16;
constexpr int kMaxAtoms = 1024;

cs_status lfail(cs_ctx* c, cs_status st, const std::string& m) {
  if (c) c->err = m;
  return st;
}

#define LD_CUDA(c, expr)                                                                 \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return lfail(c, CS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));  \
  } while (0)

long long n_grid(const cs_ctx* c) {
  return (long long)c->host.n_r * c->host.n_theta * c->host.n_phi;
}

// coordinates of grid point g (order [k][j][q]) from the r, cos(theta), phi tables
__device__ __forceinline__ void grid_point(const double* __restrict__ tab, int n_r, int n_t,
                                           int n_p, long long g, double& x, double& y,
                                           double& z) {
  const int q = (int)(g % n_p);
  const long long kj = g / n_p;
  const int j = (int)(kj % n_t), k = (int)(kj / n_t);
  const double r = tab[k], t = tab[n_r + j], ph = tab[n_r + n_t + q];
  const double st = sqrt(fmax(0.0, 1.0 - t * t));
  x = r * st * cos(ph);
  y = r * st * sin(ph);
  z = r * t;
}

struct AtomArgs {
  int n_atoms, n_basis;
  const double* atoms;   // device n_atoms x 3
  const double* coef;    // device n_atoms x n_basis
  double sig[kMaxBasis];
};

// rho[g] += sum_a sum_j coef[a][j] phi_j(|x_g - a|)
__global__ void k_atom_density(AtomArgs A, const double* __restrict__ tab, int n_r, int n_t,
                               int n_p, long long ng, double* __restrict__ rho) {
  double norm[kMaxBasis], inv2s2[kMaxBasis];
  for (int j = 0; j < A.n_basis; ++j) {
    norm[j] = pow(2.0 * kPi * A.sig[j] * A.sig[j], -1.5);
    inv2s2[j] = 1.0 / (2.0 * A.sig[j] * A.sig[j]);
  }
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng;
       g += (long long)gridDim.x * blockDim.x) {
    double x, y, z;
    grid_point(tab, n_r, n_t, n_p, g, x, y, z);
    double acc = 0.0;
    for (int a = 0; a < A.n_atoms; ++a) {
      const double dx = x - A.atoms[3 * a], dy = y - A.atoms[3 * a + 1], dz = z - A.atoms[3 * a + 2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      for (int j = 0; j < A.n_basis; ++j)
        acc = fma(A.coef[a * A.n_basis + j] * norm[j], exp(-r2 * inv2s2[j]), acc);
    }
    rho[g] += acc;
  }
}

// design rows of a chunk of grid points: Aw[p][col] = sqrt(W_g) phi_j(|x_g - a|) (column-major,
// ld = rows, col = a n_basis + j), rw[p] = sqrt(W_g) target_g; rows past the grid are zero
__global__ void k_fit_design(AtomArgs A, const double* __restrict__ tab, const double* __restrict__ wkj,
                             int n_r, int n_t, int n_p, long long ng, long long g0, int rows,
                             const double* __restrict__ target, double* __restrict__ Aw,
                             double* __restrict__ rw) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= rows) return;
  const long long g = g0 + p;
  const int nc = A.n_atoms * A.n_basis;
  if (g >= ng) {
    for (int c = 0; c < nc; ++c) Aw[p + (size_t)c * rows] = 0.0;
    rw[p] = 0.0;
    return;
  }
  double x, y, z;
  grid_point(tab, n_r, n_t, n_p, g, x, y, z);
  const double sw = sqrt(wkj[g / n_p]);
  for (int a = 0; a < A.n_atoms; ++a) {
    const double dx = x - A.atoms[3 * a], dy = y - A.atoms[3 * a + 1], dz = z - A.atoms[3 * a + 2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    for (int j = 0; j < A.n_basis; ++j) {
      const double s2 = A.sig[j] * A.sig[j];
      Aw[p + (size_t)(a * A.n_basis + j) * rows] = sw * pow(2.0 * kPi * s2, -1.5) * exp(-r2 / (2.0 * s2));
    }
  }
  rw[p] = sw * target[g];
}

__global__ void k_add(double* __restrict__ acc, const double* __restrict__ x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) acc[i] += x[i];
}

// Cholesky solve of the n x n SPD system M c = b (M column-major; host)
bool chol_solve(std::vector<double> M, std::vector<double> b, int n, std::vector<double>& c) {
  for (int j = 0; j < n; ++j) {
    double d = M[j + (size_t)j * n];
    for (int k = 0; k < j; ++k) d -= M[j + (size_t)k * n] * M[j + (size_t)k * n];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    M[j + (size_t)j * n] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = M[i + (size_t)j * n];
      for (int k = 0; k < j; ++k) s -= M[i + (size_t)k * n] * M[j + (size_t)k * n];
      M[i + (size_t)j * n] = s / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= M[i + (size_t)k * n] * b[k];
    b[i] = s / M[i + (size_t)i * n];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < n; ++k) s -= M[k + (size_t)i * n] * b[k];
    b[i] = s / M[i + (size_t)i * n];
  }
  c = b;
  return true;
}

constexpr int kFitChunk = 16384;

struct FitLayout {
  size_t atoms, coef, Aw, rw, M, Mc, bvec, bc, part, total;
};

FitLayout fit_layout(int n_atoms, int n_basis) {
  FitLayout o{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (bytes + 255) & ~size_t(255);
    return at;
  };
  const size_t nc = (size_t)n_atoms * n_basis;
  o.atoms = take((size_t)n_atoms * 3 * 8);
  o.coef = take(nc * 8);
  o.Aw = take((size_t)kFitChunk * nc * 8);
  o.rw = take((size_t)kFitChunk * 8);
  o.M = take(nc * nc * 8);
  o.Mc = take(nc * nc * 8);
  o.bvec = take(nc * 8);
  o.bc = take(nc * 8);
  size_t pe = std::max(gram_partial_elems(kFitChunk, (int)nc, (int)nc),
                       gram_partial_elems(kFitChunk, (int)nc, 1));
  o.part = take(pe * 8);
  o.total = off;
  return o;
}

}  // namespace

extern "C" {

cs_status cs_atom_descriptors(int n_atoms, const double* atoms, int n_mu, const double* mu,
                              double width, double* out) {
  if (n_atoms < 1 || !atoms || n_mu < 1 || !mu || !(width > 0) || !out) return CS_ERR_ARG;
  for (int a = 0; a < n_atoms; ++a)
    for (int k = 0; k < n_mu; ++k) {
      double s = 0.0;
      for (int b = 0; b < n_atoms; ++b) {
        if (b == a) continue;
        const double dx = atoms[3 * a] - atoms[3 * b], dy = atoms[3 * a + 1] - atoms[3 * b + 1],
                     dz = atoms[3 * a + 2] - atoms[3 * b + 2];
        const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
        const double u = r - mu[k];
        s += std::exp(-u * u / (2.0 * width * width));
      }
      out[(size_t)a * n_mu + k] = s;
    }
  return CS_OK;
}

cs_status cs_atom_density(cs_ctx* c, int n_atoms, const double* atoms, int n_basis,
                          const double* sigmas, const double* coef, double* rho,
                          cs_stream stream) {
  if (!c) return CS_ERR_ARG;
  if (!c->has_device) return lfail(c, CS_ERR_STATE, "context has no device");
  if (n_atoms < 1 || n_atoms > kMaxAtoms || n_basis < 1 || n_basis > kMaxBasis || !atoms ||
      !sigmas || !coef || !rho)
    return lfail(c, CS_ERR_ARG, "cs_atom_density: bad arguments");
  LD_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  double* buf = nullptr;
  const size_t na = (size_t)n_atoms * 3, nc = (size_t)n_atoms * n_basis;
  LD_CUDA(c, cudaMalloc((void**)&buf, (na + nc) * 8));
  LD_CUDA(c, cudaMemcpyAsync(buf, atoms, na * 8, cudaMemcpyHostToDevice, st));
  LD_CUDA(c, cudaMemcpyAsync(buf + na, coef, nc * 8, cudaMemcpyHostToDevice, st));
  AtomArgs A{};
  A.n_atoms = n_atoms;
  A.n_basis = n_basis;
  A.atoms = buf;
  A.coef = buf + na;
  for (int j = 0; j < n_basis; ++j) A.sig[j] = sigmas[j];
  const HostTables& H = c->host;
  const long long ng = n_grid(c);
  k_atom_density<<<(unsigned)std::min<long long>((ng + 255) / 256, 4096), 256, 0, st>>>(
      A, c->grid_tab, H.n_r, H.n_theta, H.n_phi, ng, rho);
  LD_CUDA(c, cudaGetLastError());
  LD_CUDA(c, cudaStreamSynchronize(st));
  LD_CUDA(c, cudaFree(buf));
  c->launches += 1;
  return CS_OK;
}

cs_status cs_fit_workspace_bytes(const cs_ctx* c, int n_atoms, int n_basis, size_t* bytes) {
  if (!c || !bytes || n_atoms < 1 || n_basis < 1) return CS_ERR_ARG;
  *bytes = fit_layout(n_atoms, n_basis).total;
  return CS_OK;
}

cs_status cs_fit_atom_density(cs_ctx* c, int n_atoms, const double* atoms, int n_basis,
                              const double* sigmas, const double* target, double ridge,
                              double* coef, void* work, cs_stream stream) {
  if (!c) return CS_ERR_ARG;
  if (!c->has_device) return lfail(c, CS_ERR_STATE, "context has no device");
  if (n_atoms < 1 || n_atoms > kMaxAtoms || n_basis < 1 || n_basis > kMaxBasis || !atoms ||
      !sigmas || !target || !coef || !work || ridge < 0)
    return lfail(c, CS_ERR_ARG, "cs_fit_atom_density: bad arguments");
  LD_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t st = (cudaStream_t)stream;
  const FitLayout lay = fit_layout(n_atoms, n_basis);
  char* w = (char*)work;
  auto D = [&](size_t o) { return reinterpret_cast<double*>(w + o); };
  const int nc = n_atoms * n_basis;
  LD_CUDA(c, cudaMemcpyAsync(D(lay.atoms), atoms, (size_t)n_atoms * 3 * 8, cudaMemcpyHostToDevice, st));
  LD_CUDA(c, cudaMemsetAsync(D(lay.M), 0, (size_t)nc * nc * 8, st));
  LD_CUDA(c, cudaMemsetAsync(D(lay.bvec), 0, (size_t)nc * 8, st));
  AtomArgs A{};
  A.n_atoms = n_atoms;
  A.n_basis = n_basis;
  A.atoms = D(lay.atoms);
  A.coef = nullptr;
  for (int j = 0; j < n_basis; ++j) A.sig[j] = sigmas[j];
  const HostTables& H = c->host;
  const long long ng = n_grid(c);
  for (long long g0 = 0; g0 < ng; g0 += kFitChunk) {
    k_fit_design<<<(kFitChunk + 127) / 128, 128, 0, st>>>(A, c->grid_tab, c->d64.wkj, H.n_r,
                                                          H.n_theta, H.n_phi, ng, g0, kFitChunk,
                                                          target, D(lay.Aw), D(lay.rw));
    LD_CUDA(c, cudaGetLastError());
    LD_CUDA(c, launch_gram<double>(D(lay.Aw), kFitChunk, D(lay.Aw), kFitChunk, kFitChunk, nc, nc,
                                   D(lay.Mc), nc, D(lay.part), st));
    LD_CUDA(c, launch_gram<double>(D(lay.Aw), kFitChunk, D(lay.rw), kFitChunk, kFitChunk, nc, 1,
                                   D(lay.bc), nc, D(lay.part), st));
    k_add<<<(nc * nc + 255) / 256, 256, 0, st>>>(D(lay.M), D(lay.Mc), nc * nc);
    k_add<<<(nc + 255) / 256, 256, 0, st>>>(D(lay.bvec), D(lay.bc), nc);
    LD_CUDA(c, cudaGetLastError());
    c->launches += 7;
  }
  std::vector<double> M((size_t)nc * nc), b(nc), x;
  LD_CUDA(c, cudaMemcpyAsync(M.data(), D(lay.M), M.size() * 8, cudaMemcpyDeviceToHost, st));
  LD_CUDA(c, cudaMemcpyAsync(b.data(), D(lay.bvec), b.size() * 8, cudaMemcpyDeviceToHost, st));
  LD_CUDA(c, cudaStreamSynchronize(st));
  double tr = 0.0;
  for (int i = 0; i < nc; ++i) tr += M[i + (size_t)i * nc];
  for (int i = 0; i < nc; ++i) M[i + (size_t)i * nc] += ridge * tr / nc;
  if (!chol_solve(M, b, nc, x)) return lfail(c, CS_ERR_NUMERIC, "cs_fit_atom_density: normal equations not positive definite");
  std::memcpy(coef, x.data(), (size_t)nc * 8);
  return CS_OK;
}

}  // extern "C"

// ====================================================================== MLP
namespace {

__global__ void k_bias_act(float* __restrict__ Z, const float* __restrict__ b, int n, int m,
                           int act) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * m) return;
  const int j = (int)(e / n);
  const float v = Z[e] + b[j];
  Z[e] = act ? tanhf(v) : v;
}

// diff = Y - T, dY = 2 diff / (n m), partial[block] = sum of diff^2 over the block
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, long long cnt,
                      float* __restrict__ dY, float* __restrict__ partial) {
  __shared__ float red[32];
  float s = 0.f;
  const float scale = 2.f / (float)cnt;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt;
       e += (long long)gridDim.x * blockDim.x) {
    const float d = Y[e] - T[e];
    dY[e] = scale * d;
    s = fmaf(d, d, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void k_sum_partials(const float* __restrict__ p, int n, long long cnt,
                               float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += p[i];
    out[0] = s / (float)cnt;
  }
}

// d <- d * (1 - h^2)
__global__ void k_tanh_back(float* __restrict__ d, const float* __restrict__ h, long long cnt) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < cnt) d[e] *= 1.f - h[e] * h[e];
}

// gb[j] = sum_a d[a + j n] (one warp per column, fixed order)
__global__ void k_col_sum(const float* __restrict__ d, int n, int m, float* __restrict__ gb) {
  const int j = blockIdx.x;
  if (j >= m) return;
  float s = 0.f;
  for (int a = threadIdx.x; a < n; a += 32) s += d[a + (size_t)j * n];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) gb[j] = s;
}

// Wt (m x k, column-major) = W^T with W (k x m, column-major)
__global__ void k_transpose(const float* __restrict__ W, int k, int m, float* __restrict__ Wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * m) return;
  const int i = e % k, j = e / k;
  Wt[j + (size_t)i * m] = W[e];
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long cnt, float lr, float c1, float c2) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= cnt) return;
  const float gg = g[e];
  const float mm = 0.9f * m[e] + 0.1f * gg;
  const float vv = 0.999f * v[e] + 0.001f * gg * gg;
  m[e] = mm;
  v[e] = vv;
  p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
}

unsigned blocks_for(long long n) { return (unsigned)std::max<long long>(1, (n + 255) / 256); }

}  // namespace

struct cs_mlp {
  int device = 0;
  int L = 0;
  std::vector<int> dims;
  std::vector<size_t> woff, boff;  // parameter offsets (floats)
  long long np = 0;
  int max_rows = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // parameters, grads, moments
  std::vector<float*> act;  // activations per layer (max_rows x dims[l])
  float *d0 = nullptr, *d1 = nullptr, *wt = nullptr, *part = nullptr, *lossd = nullptr;
  float* gpart = nullptr;
  int t = 0;
  std::string err;
};

namespace {

cs_status mfail(cs_mlp* m, cs_status st, const std::string& msg) {
  if (m) m->err = msg;
  return st;
}

#define MLP_CUDA(m, expr)                                                                \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return mfail(m, CS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));  \
  } while (0)

constexpr int kLossBlocks = 256;

// forward pass into m->act (act[0] = X copy not kept: layer 0 input read from X)
cs_status mlp_forward(cs_mlp* m, int n, const float* X, cudaStream_t st) {
  const float* in = X;
  for (int l = 0; l < m->L; ++l) {
    const int k = m->dims[l], o = m->dims[l + 1];
    float* out = m->act[l + 1];
    MLP_CUDA(m, launch_gemm_nn<float>(in, n, m->p + m->woff[l], k, n, k, o, 1.0, 0.0, out, n, st));
    k_bias_act<<<blocks_for((long long)n * o), 256, 0, st>>>(out, m->p + m->boff[l], n, o,
                                                             l < m->L - 1 ? 1 : 0);
    MLP_CUDA(m, cudaGetLastError());
    in = out;
  }
  return CS_OK;
}

// loss and gradient into m->g (loss on the device in m->lossd)
cs_status mlp_backward(cs_mlp* m, int n, const float* X, const float* T, cudaStream_t st) {
  const int L = m->L;
  const int out_dim = m->dims[L];
  const long long cnt = (long long)n * out_dim;
  float* d = m->d0;
  k_mse<<<kLossBlocks, 256, 0, st>>>(m->act[L], T, cnt, d, m->part);
  k_sum_partials<<<1, 32, 0, st>>>(m->part, kLossBlocks, cnt, m->lossd);
  MLP_CUDA(m, cudaGetLastError());
  for (int l = L - 1; l >= 0; --l) {
    const int k = m->dims[l], o = m->dims[l + 1];
    if (l < L - 1) {
      k_tanh_back<<<blocks_for((long long)n * o), 256, 0, st>>>(d, m->act[l + 1], (long long)n * o);
      MLP_CUDA(m, cudaGetLastError());
    }
    const float* in = (l == 0) ? X : m->act[l];
    // dW (k x o) = in^T d, db = column sums of d
    MLP_CUDA(m, launch_gram<float>(in, n, d, n, n, k, o, m->g + m->woff[l], k, m->gpart, st));
    k_col_sum<<<o, 32, 0, st>>>(d, n, o, m->g + m->boff[l]);
    MLP_CUDA(m, cudaGetLastError());
    if (l > 0) {
      // d_in (n x k) = d (n x o) W^T
      k_transpose<<<blocks_for((long long)k * o), 256, 0, st>>>(m->p + m->woff[l], k, o, m->wt);
      float* dn = (d == m->d0) ? m->d1 : m->d0;
      MLP_CUDA(m, launch_gemm_nn<float>(d, n, m->wt, o, n, o, k, 1.0, 0.0, dn, n, st));
      d = dn;
    }
  }
  return CS_OK;
}

}  // namespace

extern "C" {

cs_status cs_mlp_create(int n_layers, const int* dims, const float* params, int max_rows,
                        int cuda_device, cs_mlp** out) {
  if (n_layers < 1 || !dims || !params || max_rows < 1 || !out) return CS_ERR_ARG;
  for (int l = 0; l <= n_layers; ++l)
    if (dims[l] < 1 || dims[l] > 4096) return CS_ERR_ARG;
  if (cudaSetDevice(cuda_device) != cudaSuccess) return CS_ERR_CUDA;
  cs_mlp* m = new cs_mlp;
  m->device = cuda_device;
  m->L = n_layers;
  m->dims.assign(dims, dims + n_layers + 1);
  m->max_rows = max_rows;
  size_t off = 0;
  int widest = 0;
  for (int l = 0; l < n_layers; ++l) {
    m->woff.push_back(off);
    off += (size_t)dims[l] * dims[l + 1];
    m->boff.push_back(off);
    off += dims[l + 1];
    widest = std::max(widest, std::max(dims[l], dims[l + 1]));
  }
  m->np = (long long)off;
  size_t pe = 0;
  for (int l = 0; l < n_layers; ++l)
    pe = std::max(pe, gram_partial_elems(max_rows, dims[l], dims[l + 1]));
  bool ok = true;
  for (float** q : {&m->p, &m->g, &m->m, &m->v})
    ok = ok && cudaMalloc((void**)q, off * sizeof(float)) == cudaSuccess;
  m->act.assign(n_layers + 1, nullptr);
  for (int l = 1; l <= n_layers; ++l)
    ok = ok && cudaMalloc((void**)&m->act[l], (size_t)max_rows * dims[l] * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void**)&m->d0, (size_t)max_rows * widest * sizeof(float)) == cudaSuccess &&
       cudaMalloc((void**)&m->d1, (size_t)max_rows * widest * sizeof(float)) == cudaSuccess &&
       cudaMalloc((void**)&m->wt, (size_t)widest * widest * sizeof(float)) == cudaSuccess &&
       cudaMalloc((void**)&m->part, kLossBlocks * sizeof(float)) == cudaSuccess &&
       cudaMalloc((void**)&m->lossd, sizeof(float)) == cudaSuccess &&
       cudaMalloc((void**)&m->gpart, std::max<size_t>(pe, 1) * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cs_mlp_free(m);
    return CS_ERR_ALLOC;
  }
  if (cudaMemcpy(m->p, params, off * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m, 0, off * sizeof(float)) != cudaSuccess ||
      cudaMemset(m->v, 0, off * sizeof(float)) != cudaSuccess) {
    cs_mlp_free(m);
    return CS_ERR_CUDA;
  }
  *out = m;
  return CS_OK;
}

cs_status cs_mlp_free(cs_mlp* m) {
  if (!m) return CS_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  for (float* q : {m->p, m->g, m->m, m->v, m->d0, m->d1, m->wt, m->part, m->lossd, m->gpart})
    if (q) cudaFree(q);
  for (float* q : m->act)
    if (q) cudaFree(q);
  delete m;
  return CS_OK;
}

cs_status cs_mlp_param_count(const cs_mlp* m, long long* count) {
  if (!m || !count) return CS_ERR_ARG;
  *count = m->np;
  return CS_OK;
}

cs_status cs_mlp_params(const cs_mlp* m, float* params) {
  if (!m || !params) return CS_ERR_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return CS_ERR_CUDA;
  if (cudaMemcpy(params, m->p, m->np * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return CS_ERR_CUDA;
  return CS_OK;
}

cs_status cs_mlp_forward(cs_mlp* m, int n, const float* X, float* Y, cs_stream stream) {
  if (!m || n < 1 || n > m->max_rows || !X || !Y) return mfail(m, CS_ERR_ARG, "cs_mlp_forward: bad arguments");
  MLP_CUDA(m, cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  cs_status s = mlp_forward(m, n, X, st);
  if (s != CS_OK) return s;
  MLP_CUDA(m, cudaMemcpyAsync(Y, m->act[m->L], (size_t)n * m->dims[m->L] * sizeof(float),
                              cudaMemcpyDeviceToDevice, st));
  return CS_OK;
}

cs_status cs_mlp_loss_grad(cs_mlp* m, int n, const float* X, const float* T, float* loss,
                           float* grads, cs_stream stream) {
  if (!m || n < 1 || n > m->max_rows || !X || !T) return mfail(m, CS_ERR_ARG, "cs_mlp_loss_grad: bad arguments");
  MLP_CUDA(m, cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  cs_status s = mlp_forward(m, n, X, st);
  if (s != CS_OK) return s;
  if ((s = mlp_backward(m, n, X, T, st)) != CS_OK) return s;
  if (loss) MLP_CUDA(m, cudaMemcpyAsync(loss, m->lossd, sizeof(float), cudaMemcpyDeviceToHost, st));
  if (grads) MLP_CUDA(m, cudaMemcpyAsync(grads, m->g, m->np * sizeof(float), cudaMemcpyDeviceToHost, st));
  MLP_CUDA(m, cudaStreamSynchronize(st));
  return CS_OK;
}

cs_status cs_mlp_train_step(cs_mlp* m, int n, const float* X, const float* T, float lr,
                            float* loss, cs_stream stream) {
  if (!m || n < 1 || n > m->max_rows || !X || !T || !(lr > 0)) return mfail(m, CS_ERR_ARG, "cs_mlp_train_step: bad arguments");
  MLP_CUDA(m, cudaSetDevice(m->device));
  cudaStream_t st = (cudaStream_t)stream;
  cs_status s = mlp_forward(m, n, X, st);
  if (s != CS_OK) return s;
  if ((s = mlp_backward(m, n, X, T, st)) != CS_OK) return s;
  m->t += 1;
  const float c1 = 1.f - std::pow(0.9f, (float)m->t), c2 = 1.f - std::pow(0.999f, (float)m->t);
  k_adam<<<blocks_for(m->np), 256, 0, st>>>(m->p, m->g, m->m, m->v, m->np, lr, c1, c2);
  MLP_CUDA(m, cudaGetLastError());
  if (loss) {
    MLP_CUDA(m, cudaMemcpyAsync(loss, m->lossd, sizeof(float), cudaMemcpyDeviceToHost, st));
    MLP_CUDA(m, cudaStreamSynchronize(st));
  }
  return CS_OK;
}

const char* cs_mlp_last_error(const cs_mlp* m) { return m ? m->err.c_str() : ""; }

}  // extern "C"
