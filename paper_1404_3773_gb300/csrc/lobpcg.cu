// LOBPCG with the Teter-Payne-Allan preconditioner (Sec. 3.1, 3.1.2), FP64: cs_lobpcg.
//
// Each iteration:
//   1. residuals R = H X - X diag(theta) and their norms (read back);
//   2. W = TPA-preconditioned residuals of the active columns (those above the tolerance:
//      soft locking), made orthogonal to X and orthonormalised by two Cholesky-QR passes
//      with column scaling;
//   3. HW = H W, and the active columns of the previous directions P (with H P) orthonormalised
//      by the Cholesky factor of their Gram matrix;
//   4. Rayleigh-Ritz on S = [X, W, P]: U = D R^{-1} from the overlap S^T S (so that
//      U^T S^T S U = I), eigenpairs of U^T sym(S^T H S) U, C = U Q[:, :m];
//   5. X <- S C, H X <- H S C, P <- S[:, m:] C[m:, :], H P likewise.
// A factorisation that breaks down (status read back at the end of the iteration) discards
// the iteration and restarts from the current Ritz vectors with W and P dropped.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/cs.h"
#include "cs_internal.h"
#include "hx_kernels.cuh"

using namespace cs;

namespace {

cs_status lfail(cs_ctx* c, cs_status st, const std::string& m) {
  if (c) c->err = m;
  return st;
}

#define LB_CUDA(c, expr)                                                                 \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return lfail(c, CS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));  \
  } while (0)

// R = HX - X diag(theta) (d x m, ld = d) and norms[s] = ||R[:, s]||_2 (one block per column)
__global__ void k_lb_residual(const double* __restrict__ X, const double* __restrict__ HX,
                              const double* __restrict__ theta, long long d,
                              double* __restrict__ R, double* __restrict__ norms) {
  const int s = blockIdx.x;
  const double th = theta[s];
  const double* x = X + (size_t)s * d;
  const double* hx = HX + (size_t)s * d;
  double* r = R + (size_t)s * d;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < d; i += blockDim.x) {
    const double v = hx[i] - th * x[i];
    r[i] = v;
    acc = fma(v, v, acc);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    norms[s] = sqrt(t);
  }
}

// dst[:, j] = src[:, idx[j]] (d rows, ld = d for both)
__global__ void k_lb_gather(const double* __restrict__ src, const int* __restrict__ idx,
                            long long d, double* __restrict__ dst) {
  const int j = blockIdx.y;
  const double* s = src + (size_t)idx[j] * d;
  double* t = dst + (size_t)j * d;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d;
       i += (long long)gridDim.x * blockDim.x)
    t[i] = s[i];
}

// Teter-Payne-Allan preconditioner in place on each column y of Y (d x k, ld = d):
// ke = 1/2 sum Lambda y^2 / sum y^2, g = Lambda / ke,
// y <- (27 + 18g + 12g^2 + 8g^3) / (27 + 18g + 12g^2 + 8g^3 + 16g^4) y
__global__ void k_lb_tpa(double* __restrict__ Y, long long d, const double* __restrict__ half_lambda) {
  const int s = blockIdx.x;
  double* y = Y + (size_t)s * d;
  double a = 0.0, b = 0.0;
  for (long long i = threadIdx.x; i < d; i += blockDim.x) {
    const double v = y[i];
    a = fma(half_lambda[i] * v, v, a);  // 1/2 Lambda y^2
    b = fma(v, v, b);
  }
  __shared__ double ra[32], rb[32];
  __shared__ double ke_sh;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    ra[threadIdx.x >> 5] = a;
    rb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += ra[w];
      tb += rb[w];
    }
    ke_sh = ta / tb;
  }
  __syncthreads();
  const double ke = ke_sh;
  for (long long i = threadIdx.x; i < d; i += blockDim.x) {
    const double g = 2.0 * half_lambda[i] / ke;
    const double num = 27.0 + g * (18.0 + g * (12.0 + 8.0 * g));
    const double g2 = g * g;
    y[i] *= num / (num + 16.0 * g2 * g2);
  }
}

struct LbLayout {
  size_t S, HS, Xn, HXn, Pn, HPn, R, tmp;    // d-row blocks
  size_t G1, M, U, T1, Gp, Q, Cm, U2;        // small (3m)^2
  size_t eigw, cholw, part, norms, theta, th2, idx, status, hxw;
  size_t total;
};

LbLayout lb_layout(const cs_ctx* c, int m) {
  LbLayout o{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (bytes + 255) & ~size_t(255);
    return at;
  };
  const size_t d = (size_t)c->host.d, n3 = 3 * (size_t)m;
  o.S = take(d * n3 * 8);
  o.HS = take(d * n3 * 8);
  o.Xn = take(d * m * 8);
  o.HXn = take(d * m * 8);
  o.Pn = take(d * m * 8);
  o.HPn = take(d * m * 8);
  o.R = take(d * m * 8);
  o.tmp = take(d * n3 * 8);
  o.G1 = take(n3 * n3 * 8);
  o.M = take(n3 * n3 * 8);
  o.U = take(n3 * n3 * 8);
  o.T1 = take(n3 * n3 * 8);
  o.Gp = take(n3 * n3 * 8);
  o.Q = take(n3 * n3 * 8);
  o.Cm = take(n3 * m * 8);
  o.U2 = take(n3 * n3 * 8);
  o.eigw = take((8 * n3 * n3 + 3 * n3 + 4) * 8);
  o.cholw = take((n3 * n3 + 2 * n3) * 8);
  // the partial buffer of a Gram grows with the number of row chunks, which is larger for
  // narrow products: size it for every shape up to 3m x 3m
  size_t pe = 0;
  for (int na = 1; na <= (int)n3; ++na)
    for (int nb = 1; nb <= (int)n3; ++nb)
      pe = std::max(pe, gram_partial_elems((long long)d, na, nb));
  o.part = take(pe * 8);
  o.norms = take((size_t)m * 8);
  o.theta = take(n3 * 8);
  o.th2 = take((size_t)m * 8);
  o.idx = take((size_t)m * 4);
  o.status = take(16 * 4);
  size_t hw = 0;
  cs_workspace_bytes(c, m, CS_FP64, &hw);
  o.hxw = take(hw);
  o.total = off;
  return o;
}

}  // namespace

extern "C" {

cs_status cs_lobpcg_workspace_bytes(const cs_ctx* c, int n_s, size_t* bytes) {
  if (!c || !bytes || n_s < 1) return CS_ERR_ARG;
  *bytes = lb_layout(c, n_s).total;
  return CS_OK;
}

cs_status cs_lobpcg(cs_ctx* c, int m, int n_want, double* X, long long ld, double tol,
                    int max_iter, int precondition, double* theta, double* resid, int* iters,
                    int* restarts, void* work, cs_stream stream) {
  if (!c) return CS_ERR_ARG;
  if (!c->has_device) return lfail(c, CS_ERR_STATE, "context has no device");
  if (m < 1 || n_want < 1 || n_want > m || !X || ld < c->host.d || !theta || !resid || !work ||
      max_iter < 0)
    return lfail(c, CS_ERR_ARG, "cs_lobpcg: bad arguments");
  if (!c->has_potential) return lfail(c, CS_ERR_STATE, "cs_set_potential has not been called");
  LB_CUDA(c, cudaSetDevice(c->device));
  const long long d = c->host.d;
  const LbLayout lay = lb_layout(c, m);
  char* w = (char*)work;
  auto D = [&](size_t off) { return reinterpret_cast<double*>(w + off); };
  double *S = D(lay.S), *HS = D(lay.HS), *Xn = D(lay.Xn), *HXn = D(lay.HXn), *Pn = D(lay.Pn),
         *HPn = D(lay.HPn), *R = D(lay.R), *tmp = D(lay.tmp);
  double *G1 = D(lay.G1), *Mm = D(lay.M), *U = D(lay.U), *T1 = D(lay.T1), *Gp = D(lay.Gp),
         *Q = D(lay.Q), *Cm = D(lay.Cm), *U2 = D(lay.U2);
  double *eigw = D(lay.eigw), *cholw = D(lay.cholw), *part = D(lay.part), *nrm = D(lay.norms),
         *th = D(lay.theta);
  int* idx = reinterpret_cast<int*>(w + lay.idx);
  int* status = reinterpret_cast<int*>(w + lay.status);
  void* hxw = w + lay.hxw;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned gx = (unsigned)std::min<long long>((d + 255) / 256, 1024);
  auto applyH = [&](const double* in, double* out, int n) -> cs_status {
    return cs_apply_H(c, n, in, out, d, CS_FP64, hxw, stream);
  };
  // C = A^T B for d-row blocks (ld = lda = ldb = d) or small matrices
  auto gram = [&](const double* A, long long lda, const double* B, long long ldb, long long rows,
                  int na, int nb, double* C) {
    return launch_gram<double>(A, lda, B, ldb, rows, na, nb, C, na, part, st);
  };
  auto gemm = [&](const double* A, long long lda, const double* Qm, int ldq, long long rows,
                  int k, int n, double alpha, double beta, double* C, long long ldc) {
    return launch_gemm_nn<double>(A, lda, Qm, ldq, rows, k, n, alpha, beta, C, ldc, st);
  };
  // ---- start: X <- CholQR2(X) into S[:, :m], HX into HS[:, :m], Rayleigh-Ritz
  LB_CUDA(c, launch_copy_block<double>(X, ld, S, d, d, m, st));
  for (int pass = 0; pass < 2; ++pass) {
    LB_CUDA(c, gram(S, d, S, d, d, m, m, Mm));
    LB_CUDA(c, launch_cholqr_factor(Mm, m, U, cholw, status + pass, st));
    LB_CUDA(c, gemm(S, d, U, m, d, m, m, 1.0, 0.0, tmp, d));
    LB_CUDA(c, launch_copy_block<double>(tmp, d, S, d, d, m, st));
  }
  cs_status s = applyH(S, HS, m);
  if (s != CS_OK) return s;
  LB_CUDA(c, gram(S, d, HS, d, d, m, m, G1));
  LB_CUDA(c, launch_sym_eig(G1, m, th, Q, eigw, status + 2, st));
  LB_CUDA(c, gemm(S, d, Q, m, d, m, m, 1.0, 0.0, tmp, d));
  LB_CUDA(c, launch_copy_block<double>(tmp, d, S, d, d, m, st));
  LB_CUDA(c, gemm(HS, d, Q, m, d, m, m, 1.0, 0.0, tmp, d));
  LB_CUDA(c, launch_copy_block<double>(tmp, d, HS, d, d, m, st));
  c->launches += 14;
  int hs[16];
  LB_CUDA(c, cudaMemcpyAsync(hs, status, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
  LB_CUDA(c, cudaStreamSynchronize(st));
  if (hs[0] != 0 || hs[1] != 0) return lfail(c, CS_ERR_CHOLESKY, "cs_lobpcg: initial block is rank deficient");
  if (hs[2] < 0) return lfail(c, CS_ERR_NOT_CONVERGED, "cs_lobpcg: eigensolver did not converge");
  bool haveP = false;
  int it = 0, nrest = 0;
  std::vector<double> hn(m), hth(m);  // residual norms; Ritz values of the last accepted step
  LB_CUDA(c, cudaMemcpy(hth.data(), th, m * 8, cudaMemcpyDeviceToHost));
  std::vector<int> act;
  cs_status result = CS_ERR_NOT_CONVERGED;
  for (;; ++it) {
    // 1. residuals
    k_lb_residual<<<m, 256, 0, st>>>(S, HS, th, d, R, nrm);
    LB_CUDA(c, cudaGetLastError());
    c->launches += 1;
    LB_CUDA(c, cudaMemcpyAsync(hn.data(), nrm, m * 8, cudaMemcpyDeviceToHost, st));
    LB_CUDA(c, cudaStreamSynchronize(st));
    double worst = 0.0;
    for (int i = 0; i < n_want; ++i) worst = std::max(worst, hn[i]);
    if (worst <= tol) {
      result = CS_OK;
      break;
    }
    if (it >= max_iter) break;
    act.clear();
    for (int i = 0; i < m; ++i)
      if (hn[i] > tol) act.push_back(i);
    const int k = (int)act.size();
    LB_CUDA(c, cudaMemcpyAsync(idx, act.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
    double* Wb = S + (size_t)m * d;
    double* HWb = HS + (size_t)m * d;
    // 2. W = T R_active, orthogonal to X, CholQR2
    k_lb_gather<<<dim3(gx, k), 256, 0, st>>>(R, idx, d, Wb);
    LB_CUDA(c, cudaGetLastError());
    if (precondition) {
      k_lb_tpa<<<k, 256, 0, st>>>(Wb, d, c->d64.half_lambda);
      LB_CUDA(c, cudaGetLastError());
    }
    LB_CUDA(c, gram(S, d, Wb, d, d, m, k, T1));                  // X^T W (m x k)
    LB_CUDA(c, gemm(S, d, T1, m, d, m, k, -1.0, 1.0, Wb, d));    // W -= X (X^T W)
    for (int pass = 0; pass < 2; ++pass) {
      LB_CUDA(c, gram(Wb, d, Wb, d, d, k, k, Mm));
      LB_CUDA(c, launch_cholqr_factor(Mm, k, U, cholw, status + pass, st));
      LB_CUDA(c, gemm(Wb, d, U, k, d, k, k, 1.0, 0.0, tmp, d));
      LB_CUDA(c, launch_copy_block<double>(tmp, d, Wb, d, d, k, st));
    }
    c->launches += 12;
    // 3. H W, and the active previous directions
    if ((s = applyH(Wb, HWb, k)) != CS_OK) return s;
    int n = m + k;
    if (haveP) {
      double* Pb = S + (size_t)(m + k) * d;
      double* HPb = HS + (size_t)(m + k) * d;
      k_lb_gather<<<dim3(gx, k), 256, 0, st>>>(Pn, idx, d, tmp);
      k_lb_gather<<<dim3(gx, k), 256, 0, st>>>(HPn, idx, d, tmp + (size_t)k * d);
      LB_CUDA(c, cudaGetLastError());
      LB_CUDA(c, gram(tmp, d, tmp, d, d, k, k, Mm));
      LB_CUDA(c, launch_cholqr_factor(Mm, k, U, cholw, status + 2, st));
      LB_CUDA(c, gemm(tmp, d, U, k, d, k, k, 1.0, 0.0, Pb, d));
      LB_CUDA(c, gemm(tmp + (size_t)k * d, d, U, k, d, k, k, 1.0, 0.0, HPb, d));
      c->launches += 6;
      n += k;
    } else {
      LB_CUDA(c, cudaMemsetAsync(status + 2, 0, sizeof(int), st));
    }
    // 4. Rayleigh-Ritz on S = [X, W, P]
    LB_CUDA(c, gram(S, d, HS, d, d, n, n, G1));                  // S^T H S
    LB_CUDA(c, gram(S, d, S, d, d, n, n, Mm));                   // S^T S
    LB_CUDA(c, launch_cholqr_factor(Mm, n, U2, cholw, status + 3, st));  // U2^T M U2 = I
    LB_CUDA(c, gemm(G1, n, U2, n, n, n, n, 1.0, 0.0, T1, n));    // G1 U2
    LB_CUDA(c, gram(U2, n, T1, n, n, n, n, Gp));                 // U2^T G1 U2
    LB_CUDA(c, launch_sym_eig(Gp, n, th, Q, eigw, status + 4, st));
    LB_CUDA(c, gemm(U2, n, Q, n, n, n, m, 1.0, 0.0, Cm, n));     // C = U2 Q[:, :m]
    // 5. new X, H X, P, H P
    LB_CUDA(c, gemm(S, d, Cm, n, d, n, m, 1.0, 0.0, Xn, d));
    LB_CUDA(c, gemm(HS, d, Cm, n, d, n, m, 1.0, 0.0, HXn, d));
    LB_CUDA(c, gemm(S + (size_t)m * d, d, Cm + m, n, d, n - m, m, 1.0, 0.0, Pn, d));
    LB_CUDA(c, gemm(HS + (size_t)m * d, d, Cm + m, n, d, n - m, m, 1.0, 0.0, HPn, d));
    c->launches += 11;
    LB_CUDA(c, cudaMemcpyAsync(hs, status, 5 * sizeof(int), cudaMemcpyDeviceToHost, st));
    LB_CUDA(c, cudaStreamSynchronize(st));
    const bool broke = hs[0] != 0 || hs[1] != 0 || hs[2] != 0 || hs[3] != 0 || hs[4] < 0;
    if (broke) {  // restart from the current Ritz vectors (theta and S[:, :m] unchanged)
      haveP = false;
      ++nrest;
      LB_CUDA(c, cudaMemcpyAsync(th, hth.data(), m * 8, cudaMemcpyHostToDevice, st));
      continue;
    }
    LB_CUDA(c, launch_copy_block<double>(Xn, d, S, d, d, m, st));
    LB_CUDA(c, launch_copy_block<double>(HXn, d, HS, d, d, m, st));
    c->launches += 2;
    LB_CUDA(c, cudaMemcpyAsync(hth.data(), th, m * 8, cudaMemcpyDeviceToHost, st));
    haveP = true;
  }
  // outputs
  LB_CUDA(c, launch_copy_block<double>(S, d, X, ld, d, m, st));
  LB_CUDA(c, cudaMemcpyAsync(theta, th, m * 8, cudaMemcpyDeviceToDevice, st));
  LB_CUDA(c, cudaMemcpyAsync(resid, nrm, m * 8, cudaMemcpyDeviceToDevice, st));
  LB_CUDA(c, cudaStreamSynchronize(st));
  if (iters) *iters = it;
  if (restarts) *restarts = nrest;
  if (result != CS_OK) return lfail(c, CS_ERR_NOT_CONVERGED, "cs_lobpcg: tolerance not reached");
  return CS_OK;
}

}  // extern "C"
