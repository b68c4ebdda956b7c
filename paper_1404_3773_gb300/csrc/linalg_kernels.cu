// Dense FP64 pieces of the ChFSI iteration (Sec. 3.2.1): Gram matrices and block
// rotations for Cholesky-QR (Sec. 3.1.1: Cholesky after column scaling) and Rayleigh-
// Ritz, a one-CTA parallel cyclic Jacobi eigensolver for the projected matrix, residual
// norms, conversions and small vector helpers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <utility>

#include "df64.cuh"
#include "hx_kernels.cuh"

namespace cs {

// ------------------------------------------------------------------ Gram  C = A^T B
// Tiles of (16U) x (16U) outputs, U <= 6 picked from n so that 80 states are one tile; the
// d rows are split into chunks so that about two CTAs run per SM; partial products of the
// chunks are summed in a fixed order (deterministic).
constexpr int GK = 16;      // rows of d per step
constexpr int kTargetCtas = 2 * 152;

static int tile_u(int n) {
  int tiles = (n + 95) / 96;
  int u = (n + 16 * tiles - 1) / (16 * tiles);
  return u < 1 ? 1 : (u > 6 ? 6 : u);
}

static void gram_shape(long long d, int na, int nb, int& u, int& ta, int& tb, int& chunks,
                       long long& rows) {
  u = tile_u(na > nb ? na : nb);
  ta = (na + 16 * u - 1) / (16 * u);
  tb = (nb + 16 * u - 1) / (16 * u);
  int want = kTargetCtas / (ta * tb);
  if (want < 1) want = 1;
  rows = (d + want - 1) / want;
  rows = ((rows + GK - 1) / GK) * GK;
  if (rows < GK) rows = GK;
  chunks = (int)((d + rows - 1) / rows);
}

size_t gram_partial_elems(long long d, int na, int nb) {
  int u, ta, tb, chunks;
  long long rows;
  gram_shape(d, na, nb, u, ta, tb, chunks, rows);
  return (size_t)chunks * (size_t)na * (size_t)nb;
}

// storage value of a compute-type accumulator
__device__ __forceinline__ double out_val(double v) { return v; }
__device__ __forceinline__ float out_val(float v) { return v; }
__device__ __forceinline__ double out_val(df64 v) { return v.to_double(); }

// F: storage type of A, B and the partials; C: arithmetic (F, or df64 for F = double)
template <typename F, typename C, int U>
__global__ void __launch_bounds__(256) k_gram_partial(const F* __restrict__ A, long long lda,
                                                       const F* __restrict__ B,
                                                       long long ldb, long long d, int na,
                                                       int nb, long long rows,
                                                       F* __restrict__ partial) {
  constexpr int T = 16 * U;
  const int i0 = blockIdx.x * T, j0 = blockIdx.y * T;
  const int chunk = blockIdx.z;
  const long long r0 = (long long)chunk * rows;
  const long long r1 = min(d, r0 + rows);
  __shared__ C As[GK][T + 1];
  __shared__ C Bs[GK][T + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  MacAcc<C> acc[U][U];
  for (long long rb = r0; rb < r1; rb += GK) {
    for (int idx = tid; idx < GK * T; idx += 256) {
      int rr = idx % GK, cc = idx / GK;
      long long r = rb + rr;
      int i = i0 + cc, j = j0 + cc;
      As[rr][cc] = (r < r1 && i < na) ? C(A[r + (long long)i * lda]) : C(0);
      Bs[rr][cc] = (r < r1 && j < nb) ? C(B[r + (long long)j * ldb]) : C(0);
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < GK; ++rr) {
      C a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = As[rr][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < U; ++v) b[v] = Bs[rr][ty + 16 * v];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v].add_prod(a[u], b[v]);
    }
    __syncthreads();
  }
  F* P = partial + (size_t)chunk * na * nb;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      int i = i0 + tx + 16 * u, j = j0 + ty + 16 * v;
      if (i < na && j < nb) P[i + (size_t)j * na] = out_val(acc[u][v].value());
    }
}

// 32 elements x 8 chunk slices per 256-thread block; slices summed in a fixed order
template <typename F>
__global__ void k_gram_reduce(const F* __restrict__ partial, int chunks, int na, int nb,
                              F* __restrict__ C, int ldc) {
  __shared__ F red[8][33];
  const int el = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + el;
  const int E = na * nb;
  F s = F(0);
  if (e < E)
    for (int c = sl; c < chunks; c += 8) s += partial[(size_t)c * E + e];
  red[sl][el] = s;
  __syncthreads();
  if (sl == 0 && e < E) {
    F t = F(0);
    for (int k = 0; k < 8; ++k) t += red[k][el];
    int i = e % na, j = e / na;
    C[i + (size_t)j * ldc] = t;
  }
}

template <typename F, typename C>
static cudaError_t gram_impl(const F* A, long long lda, const F* B, long long ldb, long long d,
                             int na, int nb, F* Cout, int ldc, F* partial, cudaStream_t stream) {
  int u, ta, tb, chunks;
  long long rows;
  gram_shape(d, na, nb, u, ta, tb, chunks, rows);
  dim3 grid(ta, tb, chunks);
  switch (u) {
    case 1: k_gram_partial<F, C, 1><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 2: k_gram_partial<F, C, 2><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 3: k_gram_partial<F, C, 3><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 4: k_gram_partial<F, C, 4><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 5: k_gram_partial<F, C, 5><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    default: k_gram_partial<F, C, 6><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
  }
  int tot = na * nb;
  k_gram_reduce<F><<<(tot + 31) / 32, 256, 0, stream>>>(partial, chunks, na, nb, Cout, ldc);
  return cudaGetLastError();
}

template <typename F>
cudaError_t launch_gram(const F* A, long long lda, const F* B, long long ldb, long long d, int na,
                        int nb, F* C, int ldc, F* partial, cudaStream_t stream) {
  return gram_impl<F, F>(A, lda, B, ldb, d, na, nb, C, ldc, partial, stream);
}

cudaError_t launch_gram_df(const double* A, long long lda, const double* B, long long ldb,
                           long long d, int na, int nb, double* C, int ldc, double* partial,
                           cudaStream_t stream) {
  return gram_impl<double, df64>(A, lda, B, ldb, d, na, nb, C, ldc, partial, stream);
}

// ------------------------------------------------------------------ C = alpha A Q + beta C
// 64 rows x (16U) columns per CTA; U from n so that 80 states are one column tile.
template <typename F, typename Cm, int U>
__global__ void __launch_bounds__(256) k_gemm_nn(const F* __restrict__ A, long long lda,
                                                  const F* __restrict__ Q, int ldq,
                                                  long long d, int K, int n, F alpha,
                                                  F beta, F* C, long long ldc) {
  constexpr int BM = 64, BN = 16 * U;
  const long long r0 = (long long)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  __shared__ Cm As[GK][BM + 1];  // As[k][r]
  __shared__ Cm Qs[GK][BN + 1];  // Qs[k][j]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  MacAcc<Cm> acc[4][U];
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int idx = tid; idx < GK * BM; idx += 256) {
      int rr = idx % BM, kk = idx / BM;
      long long r = r0 + rr;
      int k = k0 + kk;
      As[kk][rr] = (r < d && k < K) ? Cm(A[r + (long long)k * lda]) : Cm(0);
    }
    for (int idx = tid; idx < GK * BN; idx += 256) {
      int kk = idx % GK, jj = idx / GK;
      int k = k0 + kk, j = j0 + jj;
      Qs[kk][jj] = (k < K && j < n) ? Cm(Q[k + (long long)j * ldq]) : Cm(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      Cm a[4], b[U];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < U; ++v) b[v] = Qs[kk][ty + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v].add_prod(a[u], b[v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < U; ++v) {
    int j = j0 + ty + 16 * v;
    if (j >= n) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      long long r = r0 + tx + 16 * u;
      if (r >= d) continue;
      F* c = C + r + (long long)j * ldc;
      const Cm av = acc[u][v].value();
      *c = (beta == F(0)) ? out_val(Cm(alpha) * av)
                          : out_val(fma(Cm(alpha), av, Cm(beta) * Cm(*c)));
    }
  }
}

template <typename F, typename Cm>
static cudaError_t gemm_nn_impl(const F* A, long long lda, const F* Q, int ldq, long long d,
                                int k, int n, double alpha, double beta, F* C, long long ldc,
                                cudaStream_t stream) {
  const int u = tile_u(n);
  dim3 grid((unsigned)((d + 63) / 64), (n + 16 * u - 1) / (16 * u));
  switch (u) {
    case 1: k_gemm_nn<F, Cm, 1><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, (F)alpha, (F)beta, C, ldc); break;
    case 2: k_gemm_nn<F, Cm, 2><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, (F)alpha, (F)beta, C, ldc); break;
    case 3: k_gemm_nn<F, Cm, 3><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, (F)alpha, (F)beta, C, ldc); break;
    case 4: k_gemm_nn<F, Cm, 4><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, (F)alpha, (F)beta, C, ldc); break;
    case 5: k_gemm_nn<F, Cm, 5><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, (F)alpha, (F)beta, C, ldc); break;
    default: k_gemm_nn<F, Cm, 6><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, (F)alpha, (F)beta, C, ldc); break;
  }
  return cudaGetLastError();
}

template <typename F>
cudaError_t launch_gemm_nn(const F* A, long long lda, const F* Q, int ldq, long long d, int k,
                           int n, double alpha, double beta, F* C, long long ldc,
                           cudaStream_t stream) {
  return gemm_nn_impl<F, F>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc, stream);
}

cudaError_t launch_gemm_nn_df(const double* A, long long lda, const double* Q, int ldq,
                              long long d, int k, int n, double alpha, double beta, double* C,
                              long long ldc, cudaStream_t stream) {
  return gemm_nn_impl<double, df64>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc, stream);
}

template cudaError_t launch_gram<double>(const double*, long long, const double*, long long,
                                         long long, int, int, double*, int, double*,
                                         cudaStream_t);
template cudaError_t launch_gram<float>(const float*, long long, const float*, long long,
                                        long long, int, int, float*, int, float*, cudaStream_t);
template cudaError_t launch_gemm_nn<double>(const double*, long long, const double*, int,
                                            long long, int, int, double, double, double*,
                                            long long, cudaStream_t);
template cudaError_t launch_gemm_nn<float>(const float*, long long, const float*, int, long long,
                                           int, int, double, double, float*, long long,
                                           cudaStream_t);

// y[p + s ld] *= h[p]  (rows of an n_p x S block scaled by the projector couplings)
template <typename F>
__global__ void k_scale_rows(F* __restrict__ y, int n_p, int S, int ld, const F* __restrict__ h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_p * S) return;
  const int p = i % n_p, s = i / n_p;
  y[p + (size_t)s * ld] *= h[p];
}

template <typename F>
cudaError_t launch_scale_rows(F* y, int n_p, int S, int ld, const F* h, cudaStream_t stream) {
  const int n = n_p * S;
  k_scale_rows<F><<<(n + 255) / 256, 256, 0, stream>>>(y, n_p, S, ld, h);
  return cudaGetLastError();
}
template cudaError_t launch_scale_rows<double>(double*, int, int, int, const double*, cudaStream_t);
template cudaError_t launch_scale_rows<float>(float*, int, int, int, const float*, cudaStream_t);

// ------------------------------------------------------------------ Cholesky-QR factor
// From the Gram matrix M: column scaling D = diag(M)^(-1/2), D M D = L L^T, U = D R^{-1} =
// D (L^{-1})^T. Two launches:
//  1. one CTA: right-looking Cholesky, one column per step; one thread forms the pivot's
//     reciprocal square root r_j (FP64 division and square root are long-latency, and a
//     block-wide evaluation would occupy the narrow FP64 pipe) and every division is a
//     multiplication by it; L, D and r are written to `work`;
//  2. one CTA per column c of L^{-1}: forward substitution y_c = r_c, y_i = -r_i
//     sum_{k=c}^{i-1} L_ik y_k, one warp per column with the dot products split over the
//     lanes, L staged in shared memory when it fits; the columns run on separate SMs, so the
//     FP64 work spreads over the GPU instead of one SM's FP64 pipe.
template <bool SMEM>
__global__ void __launch_bounds__(1024) k_cholesky(const double* __restrict__ M, int n,
                                                    double* __restrict__ work,
                                                    int* __restrict__ status) {
  extern __shared__ double shc[];
  double* Lc = SMEM ? shc : work;                      // n x n, lower
  double* Dv = SMEM ? shc + (size_t)n * n : work + (size_t)n * n;
  double* rinv = Dv + n;                               // n: 1 / L_jj
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x, tx = tid & 31, ty = tid >> 5;
  const int nty = nt >> 5;
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    double m = M[i + (size_t)i * n];
    if (!(m > 0.0) || !isfinite(m)) {
      atomicCAS(&fail, 0, i + 1);
      Dv[i] = 0.0;
    } else {
      Dv[i] = rsqrt(m);
    }
  }
  __syncthreads();
  if (fail) {
    if (tid == 0) status[0] = fail;
    return;
  }
  for (int e = tid; e < n * n; e += nt) {
    int i = e % n, j = e / n;
    Lc[e] = (i >= j) ? Dv[i] * M[e] * Dv[j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double p = Lc[j + (size_t)j * n];
      if (!(p > 0.0) || !isfinite(p)) {
        fail = j + 1;
        rinv[j] = 0.0;
      } else {
        const double r = rsqrt(p);
        rinv[j] = r;
        Lc[j + (size_t)j * n] = p * r;
      }
    }
    __syncthreads();
    if (fail) {
      if (tid == 0) status[0] = fail;
      return;
    }
    const double r = rinv[j];
    for (int i = j + 1 + tid; i < n; i += nt) Lc[i + (size_t)j * n] *= r;
    __syncthreads();
    // trailing update of the lower triangle: warps step over columns k, lanes over rows i
    for (int k = j + 1 + ty; k < n; k += nty) {
      const double lkj = Lc[k + (size_t)j * n];
      for (int i = k + tx; i < n; i += 32) Lc[i + (size_t)k * n] -= Lc[i + (size_t)j * n] * lkj;
    }
    __syncthreads();
  }
  if (SMEM) {
    for (int e = tid; e < n * n + 2 * n; e += nt) work[e] = shc[e];
  }
  if (tid == 0) status[0] = 0;
}

template <bool SMEM>
__global__ void __launch_bounds__(32) k_tri_inv_col(const double* __restrict__ work, int n,
                                                     double* __restrict__ U,
                                                     const int* __restrict__ status) {
  extern __shared__ double shl[];
  if (status[0] != 0) return;  // the factorisation failed: U is not used
  const int c = blockIdx.x, lane = threadIdx.x;
  const double* Lg = work;
  const double* Dv = work + (size_t)n * n;
  const double* rinv = Dv + n;
  const int m = n - c;                       // rows and columns c .. n-1
  double* y = shl;                           // m
  double* Ls = shl + m;                      // m x m (SMEM): Ls[(i-c) + (k-c) m] = L[i][k]
  if (SMEM) {
    for (int e = lane; e < m * m; e += 32) {
      const int ii = e % m, kk = e / m;
      Ls[e] = (ii >= kk) ? Lg[(c + ii) + (size_t)(c + kk) * n] : 0.0;
    }
  }
  if (lane == 0) y[0] = rinv[c];
  __syncwarp();
  for (int ii = 1; ii < m; ++ii) {
    double s = 0.0;
    for (int kk = lane; kk < ii; kk += 32) {
      const double l = SMEM ? Ls[ii + (size_t)kk * m] : Lg[(c + ii) + (size_t)(c + kk) * n];
      s = fma(l, y[kk], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[ii] = -s * rinv[c + ii];
    __syncwarp();
  }
  // U[c + i n] = D_c (L^{-1})[i][c] for i >= c, zero above
  const double dc = Dv[c];
  for (int i = lane; i < n; i += 32) U[c + (size_t)i * n] = (i >= c) ? dc * y[i - c] : 0.0;
}

// The same factor for blocks whose L does not fit one CTA's shared memory, blocked over
// panels of kCholNB columns so that the O(n^3) trailing update runs on the whole GPU: per panel
// one CTA factors its diagonal block, one warp per row below it solves for the row's panel
// entries, and a grid of 32 x 32 lower tiles subtracts the panel's outer product from the
// trailing block. L lives in
// `work` (L2-resident); status is cleared before the first launch.
constexpr int kCholNB = 32;

__global__ void k_chol_init(const double* __restrict__ M, int n, double* __restrict__ work,
                            int* __restrict__ status) {
  double* Lc = work;
  double* Dv = work + (size_t)n * n;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e % n), j = (int)(e / n);
  const double mi = M[i + (size_t)i * n], mj = M[j + (size_t)j * n];
  const bool oki = mi > 0.0 && isfinite(mi), okj = mj > 0.0 && isfinite(mj);
  if (i == j) {
    Dv[i] = oki ? rsqrt(mi) : 0.0;
    if (!oki) atomicCAS(status, 0, i + 1);
  }
  Lc[e] = (i >= j && oki && okj) ? M[e] * rsqrt(mi) * rsqrt(mj) : 0.0;
}

// Panel p in two launches. The panel's 32 columns span up to n rows; one CTA updating them
// column by column was bound by one SM's FP64 pipe (161 us per panel at n = 880). Now:
//  (1) k_chol_diag: one CTA factors the 32 x 32 diagonal block in shared memory (pivot, rsqrt,
//      column scale, rank-1 update of the block's trailing lower part);
//  (2) k_chol_rows: one warp per row i below the block solves L[i][p:pe] L_D^T = A[i][p:pe] by
//      forward substitution, lane k holding column p + k of the row.
__global__ void __launch_bounds__(256) k_chol_diag(int n, int p, double* __restrict__ work,
                                                   int* __restrict__ status) {
  __shared__ double D[kCholNB][kCholNB + 1];
  __shared__ double rs[kCholNB];
  __shared__ int fail;
  double* Lc = work;
  double* rinv = work + (size_t)n * n + n;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (status[0] != 0) return;
  const int pe = min(p + kCholNB, n), nb = pe - p;
  for (int e = tid; e < nb * nb; e += nt) {
    const int i = e % nb, k = e / nb;
    D[i][k] = (i >= k) ? Lc[(p + i) + (size_t)(p + k) * n] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      fail = 0;
      const double piv = D[j][j];
      if (!(piv > 0.0) || !isfinite(piv)) {
        fail = 1;
        status[0] = p + j + 1;
      } else {
        const double r = rsqrt(piv);
        rs[j] = r;
        D[j][j] = piv * r;
      }
    }
    __syncthreads();
    if (fail) return;
    const double r = rs[j];
    for (int i = j + 1 + tid; i < nb; i += nt) D[i][j] *= r;
    __syncthreads();
    const int m = nb - j - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = j + 1 + e % m, k = j + 1 + e / m;
      if (i >= k) D[i][k] -= D[i][j] * D[k][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += nt) {
    const int i = e % nb, k = e / nb;
    if (i >= k) Lc[(p + i) + (size_t)(p + k) * n] = D[i][k];
  }
  for (int j = tid; j < nb; j += nt) rinv[p + j] = rs[j];
}

__global__ void __launch_bounds__(256) k_chol_rows(int n, int p, double* __restrict__ work,
                                                   const int* __restrict__ status) {
  if (status[0] != 0) return;
  double* Lc = work;
  const double* rinv = work + (size_t)n * n + n;
  const int pe = min(p + kCholNB, n), nb = pe - p;
  const int lane = threadIdx.x & 31;
  const long long i = pe + ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  if (i >= n) return;  // whole warps leave together
  double x = lane < nb ? Lc[i + (size_t)(p + lane) * n] : 0.0;
  for (int j = 0; j < nb; ++j) {
    // L[i][p + j] = (A[i][p + j] - sum_{k < j} L[i][p + k] L[p + j][p + k]) / L[p + j][p + j];
    // lanes k < j already hold L[i][p + k]
    const double ljk = lane < j ? Lc[(p + j) + (size_t)(p + lane) * n] : 0.0;
    double t = lane < j ? x * ljk : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const double xj = __shfl_sync(0xffffffffu, x, j);
    if (lane == j) x = (xj - t) * rinv[p + j];
  }
  if (lane < nb) Lc[i + (size_t)(p + lane) * n] = x;
}

// trailing update after panel p: L[i][k] -= sum_{j in panel} L[i][j] L[k][j], i >= k >= p + NB;
// one CTA per 32 x 32 tile on or below the diagonal (tile index t -> (ti >= tk))
__global__ void __launch_bounds__(256) k_chol_trail(int n, int p, double* __restrict__ work,
                                                    const int* __restrict__ status) {
  __shared__ double Ai[32][kCholNB + 1], Ak[32][kCholNB + 1];
  if (status[0] != 0) return;
  double* Lc = work;
  const int q = p + kCholNB;  // first trailing column
  int t = blockIdx.x, ti = 0;
  while (t > ti) {  // row tile ti holds tiles tk = 0 .. ti
    t -= ti + 1;
    ++ti;
  }
  const int tk = t;
  const int i0 = q + 32 * ti, k0 = q + 32 * tk;
  const int tid = threadIdx.x;
  for (int e = tid; e < 32 * kCholNB; e += blockDim.x) {
    const int r = e % 32, c = e / 32;
    const int ii = i0 + r, kk = k0 + r;
    Ai[r][c] = ii < n ? Lc[ii + (size_t)(p + c) * n] : 0.0;
    Ak[r][c] = kk < n ? Lc[kk + (size_t)(p + c) * n] : 0.0;
  }
  __syncthreads();
  // thread: row r = tid % 32, columns c = tid / 32 + 8 u (u < 4)
  const int r = tid & 31, cb = tid >> 5;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = 0; j < kCholNB; ++j) {
    const double a = Ai[r][j];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = fma(a, Ak[cb + 8 * u][j], acc[u]);
  }
  const int i = i0 + r;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int k = k0 + cb + 8 * u;
    if (i < n && k < n && i >= k) Lc[i + (size_t)k * n] -= acc[u];
  }
}

cudaError_t launch_cholqr_factor(const double* M, int n, double* U, double* work, int* status,
                                 cudaStream_t stream) {
  size_t smem = ((size_t)n * n + 2 * n) * sizeof(double);
  cudaError_t e;
  if (smem <= 200 * 1024) {
    e = cudaFuncSetAttribute(k_cholesky<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_cholesky<true><<<1, 1024, smem, stream>>>(M, n, work, status);
  } else {
    if ((e = cudaMemsetAsync(status, 0, sizeof(int), stream)) != cudaSuccess) return e;
    const long long n2 = (long long)n * n;
    k_chol_init<<<(unsigned)((n2 + 255) / 256), 256, 0, stream>>>(M, n, work, status);
    for (int p = 0; p < n; p += kCholNB) {
      k_chol_diag<<<1, 256, 0, stream>>>(n, p, work, status);
      const int below = n - min(p + kCholNB, n);
      if (below > 0)
        k_chol_rows<<<(unsigned)(((long long)below * 32 + 255) / 256), 256, 0, stream>>>(n, p, work,
                                                                                        status);
      const int rest = n - (p + kCholNB);
      if (rest > 0) {
        const int t = (rest + 31) / 32;
        k_chol_trail<<<(unsigned)(t * (t + 1) / 2), 256, 0, stream>>>(n, p, work, status);
      }
    }
  }
  const size_t sm2 = ((size_t)n * n + n) * sizeof(double);
  if (sm2 <= 200 * 1024) {
    e = cudaFuncSetAttribute(k_tri_inv_col<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm2);
    if (e != cudaSuccess) return e;
    k_tri_inv_col<true><<<n, 32, sm2, stream>>>(work, n, U, status);
  } else {
    k_tri_inv_col<false><<<n, 32, (size_t)n * sizeof(double), stream>>>(work, n, U, status);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ symmetric eigensolver
// One CTA, for the Rayleigh-Ritz matrix (Sec. 3.2.1) and the Lanczos tridiagonal:
//  1. Householder reduction of sym(A) to tridiagonal form T = Q^T A Q: for k = 0 .. n-3,
//     v = x - alpha e_1 (x = A[k+1:, k], alpha = -sign(x_0) |x|), v /= |v|, p = A v,
//     w = p - (v.p) v, A <- A - 2 (v w^T + w v^T) on the trailing block;
//  2. Q accumulated from the reflectors (applied in reverse order to the identity);
//  3. implicit QL iterations with a Wilkinson-type shift on (d, e): one thread generates the
//     plane rotations of an iteration, then every thread applies them, in order, to its
//     own row of Z (initially Q), so the columns of Z become the eigenvectors;
//  4. eigenvalues sorted ascending with their vectors.
// Working matrices in shared memory when they fit (n <= 112), else in `work`.
template <typename T>
struct EigEps;
template <>
struct EigEps<float> {
  static __device__ float v() { return 1.1920929e-7f; }
};
template <>
struct EigEps<double> {
  static __device__ double v() { return 2.220446049250313e-16; }
};

template <typename T, bool SMEM, bool BISECT>
__global__ void __launch_bounds__(1024) k_sym_eig(const double* __restrict__ Ain, int n,
                                                   double* __restrict__ theta,
                                                   double* __restrict__ Vout,
                                                   T* __restrict__ work,
                                                   int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char she_raw[];
  T* she = reinterpret_cast<T*>(she_raw);
  const int tid = threadIdx.x, nt = blockDim.x;
  T* A = SMEM ? she : work;                                  // n x n
  T* Z = SMEM ? she + (size_t)n * n : work + (size_t)n * n;  // n x n
  T* small = SMEM ? she + 2 * (size_t)n * n : work + 2 * (size_t)n * n;
  T* d = small;           // n
  T* e = d + n;           // n
  T* vv = e + n;          // n   Householder vector
  T* pw = vv + n;         // n   p, then w
  T* rc = pw + n;         // n   rotation cosines
  T* rs = rc + n;         // n   rotation sines
  T* dsort = rs + n;      // n
  __shared__ T red[32];
  __shared__ int ctl[4];  // 0: rotation count, 1: failure flag, 2: m, 3: converged

  auto block_sum = [&](T v) -> T {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    T t = T(0);
    const int nw = (nt + 31) / 32;
    for (int w = 0; w < nw; ++w) t += red[w];
    return t;
  };

  for (int idx = tid; idx < n * n; idx += nt) {
    int i = idx % n, j = idx / n;
    A[idx] = (T)(0.5 * (Ain[i + (size_t)j * n] + Ain[j + (size_t)i * n]));
  }
  if (tid == 0) ctl[1] = 0;
  __syncthreads();

  // 1. tridiagonalisation; reflector k is kept in A[k+1:, k] (unit vector), alpha in e[k]
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;  // length of x
    T xs = T(0);
    for (int i = tid; i < m; i += nt) {
      T x = A[(k + 1 + i) + (size_t)k * n];
      xs += x * x;
    }
    const T xnorm = sqrt(block_sum(xs));
    const T x0 = A[(k + 1) + (size_t)k * n];
    const T alpha = (x0 >= T(0)) ? -xnorm : xnorm;
    // |v|^2 = |x|^2 - 2 alpha x0 + alpha^2 = 2 (|x|^2 - alpha x0)
    const T vnorm2 = T(2) * (xnorm * xnorm - alpha * x0);
    const bool skip = !(vnorm2 > T(0));
    const T inv = skip ? T(0) : rsqrt(vnorm2);
    for (int i = tid; i < m; i += nt) {
      T x = A[(k + 1 + i) + (size_t)k * n];
      vv[i] = skip ? T(0) : (i == 0 ? x - alpha : x) * inv;
    }
    __syncthreads();
    if (skip) {
      if (tid == 0) {
        e[k] = x0;
        for (int i = 0; i < m; ++i) A[(k + 1 + i) + (size_t)k * n] = T(0);
      }
      __syncthreads();
      continue;
    }
    // p = A_sub v  (trailing block rows/cols k+1 .. n-1)
    T kp = T(0);
    for (int i = tid; i < m; i += nt) {
      T s = T(0);
      for (int j = 0; j < m; ++j) s += A[(k + 1 + i) + (size_t)(k + 1 + j) * n] * vv[j];
      pw[i] = s;
      kp += vv[i] * s;
    }
    const T K = block_sum(kp);
    for (int i = tid; i < m; i += nt) pw[i] -= K * vv[i];
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += nt) {
      int i = idx % m, j = idx / m;
      A[(k + 1 + i) + (size_t)(k + 1 + j) * n] -= T(2) * (vv[i] * pw[j] + pw[i] * vv[j]);
    }
    __syncthreads();
    // keep the reflector in column k below the subdiagonal slot
    for (int i = tid; i < m; i += nt) A[(k + 1 + i) + (size_t)k * n] = vv[i];
    if (tid == 0) e[k] = alpha;
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) d[i] = A[i + (size_t)i * n];
  if (tid == 0) {
    if (n >= 2) e[n - 2] = A[(n - 1) + (size_t)(n - 2) * n];
    e[n - 1] = T(0);  // (entries k < n-2 are the alphas stored above)
  }
  __syncthreads();
  // 2. Z = H_0 H_1 ... H_{n-3}: start from I, apply reflectors in reverse order
  for (int idx = tid; idx < n * n; idx += nt) Z[idx] = ((idx % n) == (idx / n)) ? T(1) : T(0);
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nwarps = (nt + 31) / 32;
  for (int k = n - 3; k >= 0; --k) {
    const int m = n - k - 1;
    const T* vk = A + (k + 1) + (size_t)k * n;
    for (int j = warp; j < n; j += nwarps) {  // one warp per column, lanes over rows
      T* zc = Z + (k + 1) + (size_t)j * n;
      T t = T(0);
      for (int i = lane; i < m; i += 32) t += vk[i] * zc[i];
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      t *= T(2);
      for (int i = lane; i < m; i += 32) zc[i] -= t * vk[i];
    }
    __syncthreads();
  }
  const T eps = EigEps<T>::v();
  if constexpr (BISECT) {
    // 3'. eigenvalues of the tridiagonal T = (d, e) by bisection on Sturm counts, one thread
    //     per eigenvalue (independent), eigenvectors of T by inverse iteration with the
    //     LDL^T factors of T - lambda I, Gram-Schmidt inside clusters of close eigenvalues,
    //     then Z <- Z Y. The serial chains are n steps long instead of QL's n sweeps.
    T* Y = dsort + n;              // n x n, column i: eigenvector of T for lambda_i
    T* Ls = Y + (size_t)n * n;     // n x n, column i: L factors of thread i
    T* e2 = rc;                    // e_j^2
    T* lam = rs;                   // eigenvalues, ascending
    __shared__ T bnd[2];
    for (int j = tid; j < n; j += nt) e2[j] = (j < n - 1) ? e[j] * e[j] : T(0);
    if (tid == 0) {
      T lo = d[0], hi = d[0];
      for (int j = 0; j < n; ++j) {
        const T r = (j > 0 ? fabs(e[j - 1]) : T(0)) + (j < n - 1 ? fabs(e[j]) : T(0));
        lo = fmin(lo, d[j] - r);
        hi = fmax(hi, d[j] + r);
      }
      bnd[0] = lo;
      bnd[1] = hi;
    }
    __syncthreads();
    const T glo = bnd[0], ghi = bnd[1];
    const T tnorm = fmax(fabs(glo), fabs(ghi)) + T(1e-30);
    const T piv = eps * tnorm;  // pivot guard of the Sturm and LDL^T recurrences
    for (int i = tid; i < n; i += nt) {
      T a = glo - piv, b = ghi + piv;  // count(a) <= i < count(b)
      for (int it = 0; it < 64; ++it) {
        const T x = T(0.5) * (a + b);
        if (!(x > a && x < b)) break;
        int cnt = 0;
        T q = d[0] - x;
        if (fabs(q) < piv) q = -piv;
        cnt += (q < T(0));
        for (int j = 1; j < n; ++j) {
          q = d[j] - x - e2[j - 1] / q;
          if (fabs(q) < piv) q = -piv;
          cnt += (q < T(0));
        }
        if (cnt > i) b = x;
        else a = x;
      }
      const T x = T(0.5) * (a + b);
      lam[i] = x;
      T* y = Y + (size_t)i * n;
      T* L = Ls + (size_t)i * n;
      // start vector differing per eigenvalue, so that a cluster's members start apart
      for (int j = 0; j < n; ++j) {
        const unsigned hsh = (unsigned)(j + 1) * 2654435761u ^ (unsigned)(i + 1) * 40503u;
        y[j] = T(0.5) + (T)((hsh >> 8) & 0xffffu) * T(1.0 / 65536.0);
      }
      for (int rep = 0; rep < 3; ++rep) {
        T Dp = d[0] - x;
        if (fabs(Dp) < piv) Dp = piv;
        T zp = y[0];
        y[0] = zp / Dp;
        for (int j = 1; j < n; ++j) {
          const T l = e[j - 1] / Dp;
          L[j] = l;
          const T z = y[j] - l * zp;
          T Dj = d[j] - x - l * e[j - 1];
          if (fabs(Dj) < piv) Dj = piv;
          y[j] = z / Dj;
          zp = z;
          Dp = Dj;
        }
        for (int j = n - 2; j >= 0; --j) y[j] -= L[j + 1] * y[j + 1];
        T ss = T(0);
        for (int j = 0; j < n; ++j) ss += y[j] * y[j];
        const T sc = rsqrt(ss);
        for (int j = 0; j < n; ++j) y[j] *= sc;
      }
    }
    __syncthreads();
    // clusters of eigenvalues closer than 1e-5 |T|: modified Gram-Schmidt, twice
    int* cst = reinterpret_cast<int*>(Ls);
    __shared__ int kmax;
    if (tid == 0) {
      int start = 0, km = 0;
      for (int i = 0; i < n; ++i) {
        if (i > 0 && lam[i] - lam[i - 1] > T(1e-5) * tnorm) start = i;
        cst[i] = start;
        km = max(km, i - start);
      }
      kmax = km;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 2; ++sweep)
      for (int pos = 1; pos <= kmax; ++pos) {
        for (int i = tid; i < n; i += nt) {
          if (i - cst[i] != pos) continue;
          T* y = Y + (size_t)i * n;
          for (int jv = cst[i]; jv < i; ++jv) {
            const T* u = Y + (size_t)jv * n;
            T dot = T(0);
            for (int j = 0; j < n; ++j) dot += u[j] * y[j];
            for (int j = 0; j < n; ++j) y[j] -= dot * u[j];
          }
          T ss = T(0);
          for (int j = 0; j < n; ++j) ss += y[j] * y[j];
          const T sc = rsqrt(ss);
          for (int j = 0; j < n; ++j) y[j] *= sc;
        }
        __syncthreads();
      }
    // V = Z Y (already ascending)
    for (int idx = tid; idx < n * n; idx += nt) {
      const int r = idx % n, i = idx / n;
      T acc = T(0);
      for (int k = 0; k < n; ++k) acc += Z[r + (size_t)k * n] * Y[k + (size_t)i * n];
      Vout[idx] = (double)acc;
    }
    if (theta)
      for (int i = tid; i < n; i += nt) theta[i] = (double)lam[i];
    if (tid == 0) status[0] = 1;
    return;
  }
  // 3. implicit QL on (d, e), e[i] couples i and i+1
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      if (tid == 0) {
        int m = l;
        for (; m < n - 1; ++m) {
          T dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= eps * dd) break;
        }
        ctl[0] = 0;
        if (m != l) {
          if (iter >= 60) {
            ctl[1] = 1;
          } else {
            T g = (d[l + 1] - d[l]) / (T(2) * e[l]);
            T r = hypot(g, T(1));
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            T s = T(1), c = T(1), p = T(0);
            int i = m - 1, cnt = 0;
            bool early = false;
            for (; i >= l; --i) {
              T f = s * e[i], b = c * e[i];
              r = hypot(f, g);
              e[i + 1] = r;
              if (r == T(0)) {
                d[i + 1] -= p;
                e[m] = T(0);
                early = true;
                break;
              }
              s = f / r;
              c = g / r;
              g = d[i + 1] - p;
              r = (d[i] - g) * s + T(2) * c * b;
              p = s * r;
              d[i + 1] = g + p;
              g = c * r - b;
              rc[cnt] = c;
              rs[cnt] = s;
              ++cnt;
            }
            if (!early) {
              d[l] -= p;
              e[l] = g;
              e[m] = T(0);
            }
            ctl[0] = cnt;
            ctl[2] = m;
          }
        }
        ctl[3] = (m == l) ? 1 : 0;
      }
      __syncthreads();
      const int cnt = ctl[0], m = ctl[2];
      const bool stop = ctl[1] || ctl[3];
      __syncthreads();  // everyone has read ctl before thread 0 writes it again
      if (stop) break;
      // apply the rotations (in generation order i = m-1, m-2, ...) to each row of Z
      for (int row = tid; row < n; row += nt) {
        for (int t = 0; t < cnt; ++t) {
          const int i = m - 1 - t;
          const T c = rc[t], s = rs[t];
          const T zi = Z[row + (size_t)i * n], zi1 = Z[row + (size_t)(i + 1) * n];
          Z[row + (size_t)(i + 1) * n] = s * zi + c * zi1;
          Z[row + (size_t)i * n] = c * zi - s * zi1;
        }
      }
      __syncthreads();
    }
    const bool failed_now = ctl[1] != 0;
    __syncthreads();
    if (failed_now) break;
  }
  const bool failed = ctl[1] != 0;
  // 4. sort ascending (rank of each value, ties by index) and permute the vectors
  for (int i = tid; i < n; i += nt) dsort[i] = d[i];
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const T vi = dsort[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T vj = dsort[j];
      rank += (vj < vi) || (vj == vi && j < i);
    }
    if (theta) theta[rank] = (double)vi;
    for (int r = 0; r < n; ++r) Vout[r + (size_t)rank * n] = (double)Z[r + (size_t)i * n];
  }
  if (tid == 0) status[0] = failed ? -1 : 1;
}

// ---- FP64 refinement of an FP32 eigendecomposition (Ogita-Aishima iterative refinement
// for symmetric eigenproblems): with R = I - V^T V, S = V^T A V, lam_i = S_ii/(1 - R_ii),
// E_ij = (S_ij + lam_j R_ij)/(lam_j - lam_i) for separated pairs and R_ij/2 for pairs in a
// cluster, V <- V (I + E); each step squares the error. A pair counts as clustered when
// |lam_i - lam_j| <= max(delta, 1e3 |S_ij + lam_j R_ij|) (first-order mixing above 1e-3),
// delta = 2(|S - diag(lam)|_F + |A|_F |R|_F); clusters are finished by an exact FP64 Jacobi
// on their (small) block. The FP32 vectors are first made orthonormal to FP64 precision by
// Newton-Schulz steps V <- V (3I - V^T V)/2, so that delta starts at the FP32 error of S.
// All FP64 work here is wide (n x n GEMM tiles over many CTAs), which matters on a GPU
// whose FP64 pipe is narrow: the FP32 factorisation carries the long serial chains.

// C (n x n) = op(A) B, op(A) = A^T if TA; T x T output tiles, one element per thread. The FP64
// pipe of one SM is narrow, so n <= 256 takes 8 x 8 tiles: at n = 80 that spreads the work over
// 100 CTAs instead of 25 (16 x 16 tiles).
template <bool TA, int T>
__global__ void __launch_bounds__(T * T) k_small_gemm(const double* __restrict__ A,
                                                       const double* __restrict__ B, int n,
                                                       double* __restrict__ C) {
  __shared__ double As[T][T + 1], Bs[T][T + 1];
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;
  const int i = blockIdx.x * T + tx, j = blockIdx.y * T + ty;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += T) {
    const int ka = k0 + ty, kb = k0 + tx;
    // As[kk][ii] = op(A)[i][k], Bs[kk][jj] = B[k][j]
    As[ty][tx] = (i < n && ka < n) ? (TA ? A[ka + (size_t)i * n] : A[i + (size_t)ka * n]) : 0.0;
    Bs[tx][ty] = (j < n && kb < n) ? B[kb + (size_t)j * n] : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < T; ++kk) acc = fma(As[kk][tx], Bs[kk][ty], acc);
    __syncthreads();
  }
  if (i < n && j < n) C[i + (size_t)j * n] = acc;
}

static cudaError_t small_gemm(bool ta, const double* A, const double* B, int n, double* C,
                              cudaStream_t st) {
  if (n <= 256) {
    dim3 grid((n + 7) / 8, (n + 7) / 8);
    if (ta) k_small_gemm<true, 8><<<grid, 64, 0, st>>>(A, B, n, C);
    else k_small_gemm<false, 8><<<grid, 64, 0, st>>>(A, B, n, C);
  } else {
    dim3 grid((n + 15) / 16, (n + 15) / 16);
    if (ta) k_small_gemm<true, 16><<<grid, 256, 0, st>>>(A, B, n, C);
    else k_small_gemm<false, 16><<<grid, 256, 0, st>>>(A, B, n, C);
  }
  return cudaGetLastError();
}

// lam (n), scal[0] = delta, scal[1] = |A|_F; one CTA
__global__ void __launch_bounds__(1024) k_oa_norms(const double* __restrict__ A,
                                                    const double* __restrict__ S,
                                                    const double* __restrict__ G, int n,
                                                    double* __restrict__ lam,
                                                    double* __restrict__ scal) {
  __shared__ double red[3][32];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) lam[i] = S[i + (size_t)i * n] / G[i + (size_t)i * n];
  __syncthreads();
  double a2 = 0.0, s2 = 0.0, r2 = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e % n, j = e / n;
    const double a = A[e];
    const double sv = S[e] - (i == j ? lam[i] : 0.0);
    const double rv = (i == j ? 1.0 : 0.0) - G[e];
    a2 += a * a;
    s2 += sv * sv;
    r2 += rv * rv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = a2;
    red[1][tid >> 5] = s2;
    red[2][tid >> 5] = r2;
  }
  __syncthreads();
  if (tid == 0) {
    double ta = 0.0, ts = 0.0, tr = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) {
      ta += red[0][w];
      ts += red[1][w];
      tr += red[2][w];
    }
    scal[1] = sqrt(ta);
    scal[0] = 2.0 * (sqrt(ts) + sqrt(ta) * sqrt(tr));
  }
}

// The same norms over the whole GPU for large n (one CTA reads the three n x n matrices at a
// few tens of GB/s: 1 ms at n = 880): per-CTA partial sums part[q * gridDim + b], in a fixed
// order, then one CTA adds them in CTA order (deterministic for a given grid)
__global__ void __launch_bounds__(256) k_oa_norms_part(const double* __restrict__ A,
                                                       const double* __restrict__ S,
                                                       const double* __restrict__ G, int n,
                                                       double* __restrict__ lam,
                                                       double* __restrict__ part) {
  __shared__ double red[3][8];
  const int tid = threadIdx.x;
  const long long n2 = (long long)n * n;
  double a2 = 0.0, s2 = 0.0, r2 = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + tid; e < n2;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    const double a = A[e];
    double sv = S[e], rv = -G[e];
    if (i == j) {
      const double l = S[e] / G[e];
      lam[i] = l;
      sv -= l;
      rv += 1.0;
    }
    a2 += a * a;
    s2 += sv * sv;
    r2 += rv * rv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    r2 += __shfl_xor_sync(0xffffffffu, r2, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = a2;
    red[1][tid >> 5] = s2;
    red[2][tid >> 5] = r2;
  }
  __syncthreads();
  if (tid < 3) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[tid][w];
    part[(size_t)tid * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(32) k_oa_norms_fin(const double* __restrict__ part, int nb,
                                                     double* __restrict__ scal) {
  if (threadIdx.x != 0) return;
  double t[3];
  for (int q = 0; q < 3; ++q) {
    double v = 0.0;
    for (int b = 0; b < nb; ++b) v += part[(size_t)q * nb + b];
    t[q] = v;
  }
  scal[1] = sqrt(t[0]);
  scal[0] = 2.0 * (sqrt(t[1]) + sqrt(t[0]) * sqrt(t[2]));
}

// M = 1.5 I - 0.5 G (Newton-Schulz factor), grid over elements
__global__ void k_ns_factor(const double* __restrict__ G, int n, double* __restrict__ M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e % n, j = e / n;
  M[e] = (i == j ? 1.5 : 0.0) - 0.5 * G[e];
}

// Ep = I + E (n x n), grid over elements
__global__ void k_oa_update(const double* __restrict__ S, const double* __restrict__ G, int n,
                            const double* __restrict__ lam, const double* __restrict__ scal,
                            double* __restrict__ Ep) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e % n, j = e / n;
  const double r = (i == j ? 1.0 : 0.0) - G[e];
  double v;
  if (i == j) {
    v = 0.5 * r;
  } else {
    const double num = S[e] + lam[j] * r;
    const double dl = lam[j] - lam[i];
    const double lim = fmax(scal[0], 1e3 * fabs(num));
    v = (fabs(dl) > lim) ? num / dl : 0.5 * r;
  }
  Ep[e] = (i == j ? 1.0 : 0.0) + v;
}

// one CTA: theta_i = S_ii/G_ii; sort; clusters (consecutive gaps <= max(delta, 1e5 max|S_ij|))
// diagonalised by an exact FP64 Jacobi per cluster (one thread per cluster, blocks kept in
// Vout as scratch); then Vout = (sorted V) * blockdiag(J). scratch: 2 n^2 + 2 n doubles.
// status[0] = -2 if a cluster Jacobi did not converge (the FP32 stage leaves -1 / 1).
__global__ void __launch_bounds__(1024) k_oa_final(const double* __restrict__ S,
                                                    const double* __restrict__ G,
                                                    const double* __restrict__ V, int n,
                                                    const double* __restrict__ scal,
                                                    double* __restrict__ theta,
                                                    double* __restrict__ Vout,
                                                    double* __restrict__ scratch,
                                                    int* __restrict__ status) {
  __shared__ double red[32];
  __shared__ double dc_sh;
  const int tid = threadIdx.x, nt = blockDim.x;
  double* lam = scratch;                                       // n   sorted eigenvalues
  int* perm = reinterpret_cast<int*>(scratch + n);             // n   sorted -> original
  int* cstart = perm + n;                                      // n   first column of cluster
  double* Jb = scratch + 2 * (size_t)n;                        // n^2 (k x k blocks, ld n)
  double* Vs = Jb + (size_t)n * n;                             // n^2 sorted vectors
  double mo = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e % n, j = e / n;
    if (i != j) mo = fmax(mo, fabs(S[e]));
  }
  for (int o = 16; o > 0; o >>= 1) mo = fmax(mo, __shfl_xor_sync(0xffffffffu, mo, o));
  if ((tid & 31) == 0) red[tid >> 5] = mo;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) m = fmax(m, red[w]);
    dc_sh = fmax(scal[0], 1e3 * m);
  }
  // the unsorted Rayleigh quotients go through theta (overwritten with the sorted values at the
  // end): n divisions instead of one per pair, which cost milliseconds on one SM at n = 880
  for (int i = tid; i < n; i += nt) theta[i] = S[i + (size_t)i * n] / G[i + (size_t)i * n];
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const double vi = theta[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double vj = theta[j];
      rank += (vj < vi) || (vj == vi && j < i);
    }
    lam[rank] = vi;
    perm[rank] = i;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) {
    const int r = e % n, c = e / n;
    Vs[e] = V[r + (size_t)perm[c] * n];
  }
  const double dc = dc_sh;
  for (int c = tid; c < n; c += nt) {
    int i0 = c;
    while (i0 > 0 && lam[i0] - lam[i0 - 1] <= dc) --i0;
    cstart[c] = i0;
  }
  __syncthreads();
  bool fail = false;
  for (int i0 = tid; i0 < n; i0 += nt) {
    if (cstart[i0] != i0) continue;  // not the first column of its cluster
    int i1 = i0;
    while (i1 + 1 < n && cstart[i1 + 1] == i0) ++i1;
    const int k = i1 - i0 + 1;
    double* J = Jb + (size_t)i0 * n + i0;    // k x k, leading dimension n
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) J[a + (size_t)b * n] = (a == b) ? 1.0 : 0.0;
    if (k == 1) continue;
    double* B = Vout + (size_t)i0 * n + i0;  // cluster block of S in sorted order
    double bn = 0.0;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        const double v = S[perm[i0 + a] + (size_t)perm[i0 + b] * n];
        B[a + (size_t)b * n] = v;
        bn += v * v;
      }
    bn = sqrt(bn);
    bool done = false;
    for (int sweep = 0; sweep < 50 && !done; ++sweep) {
      int rot = 0;
      for (int p = 0; p < k; ++p)
        for (int q = p + 1; q < k; ++q) {
          const double apq = B[p + (size_t)q * n];
          if (!(fabs(apq) > 1e-15 * bn)) continue;
          ++rot;
          const double app = B[p + (size_t)p * n], aqq = B[q + (size_t)q * n];
          const double tau = (aqq - app) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
          for (int x = 0; x < k; ++x) {  // B <- G^T B (rows p, q)
            const double bp = B[p + (size_t)x * n], bq = B[q + (size_t)x * n];
            B[p + (size_t)x * n] = c * bp - s * bq;
            B[q + (size_t)x * n] = s * bp + c * bq;
          }
          for (int x = 0; x < k; ++x) {  // B <- B G, J <- J G (columns p, q)
            const double bp = B[x + (size_t)p * n], bq = B[x + (size_t)q * n];
            B[x + (size_t)p * n] = c * bp - s * bq;
            B[x + (size_t)q * n] = s * bp + c * bq;
            const double jp = J[x + (size_t)p * n], jq = J[x + (size_t)q * n];
            J[x + (size_t)p * n] = c * jp - s * jq;
            J[x + (size_t)q * n] = s * jp + c * jq;
          }
          B[p + (size_t)q * n] = 0.0;
          B[q + (size_t)p * n] = 0.0;
        }
      done = (rot == 0);
    }
    if (!done) fail = true;
    // ascending order inside the cluster (insertion sort; J's columns follow)
    for (int a = 1; a < k; ++a)
      for (int b = a; b > 0 && B[b + (size_t)b * n] < B[(b - 1) + (size_t)(b - 1) * n]; --b) {
        const double tmp = B[b + (size_t)b * n];
        B[b + (size_t)b * n] = B[(b - 1) + (size_t)(b - 1) * n];
        B[(b - 1) + (size_t)(b - 1) * n] = tmp;
        for (int x = 0; x < k; ++x) {
          const double tj = J[x + (size_t)b * n];
          J[x + (size_t)b * n] = J[x + (size_t)(b - 1) * n];
          J[x + (size_t)(b - 1) * n] = tj;
        }
      }
    for (int a = 0; a < k; ++a) lam[i0 + a] = B[a + (size_t)a * n];
  }
  if (fail) status[0] = -2;
  __syncthreads();
  // Vout[:, c] = sum over the cluster of c: Vs[:, a] J[a][c]
  for (int e = tid; e < n * n; e += nt) {
    const int r = e % n, c = e / n;
    const int i0 = cstart[c];
    int i1 = c;
    while (i1 + 1 < n && cstart[i1 + 1] == i0) ++i1;
    double acc = 0.0;
    for (int a = i0; a <= i1; ++a) acc = fma(Vs[r + (size_t)a * n], Jb[a + (size_t)c * n], acc);
    Vout[e] = acc;
  }
  for (int i = tid; i < n; i += nt) theta[i] = lam[i];
}

// ------------------------------------------------------------------ large-n first stage
// For blocks whose tridiagonal solve does not fit one CTA's shared memory (n above 112; the
// 880-state block of the 400-atom cluster) the first stage runs in FP64 as a sequence of
// device-wide kernels on global (L2-resident) arrays instead of one CTA: two launches per
// Householder step (the reflector, recomputed per CTA, with p = A v, one warp per row: the
// trailing block is symmetric, so each warp reads a contiguous column; then w = p - (v.p) v,
// recomputed per CTA, with the rank-2 update); then multisection and inverse iteration with
// one warp per eigenvalue, Gram-Schmidt inside clusters (one CTA), and all reflectors applied
// to the eigenvector block in one launch, one warp per column. FP64 here (not FP32 as in the small
// solver): in a dense band of eigenvalues (gaps near 1e-4 of the spectral range) FP32 vectors
// leave couplings that the refinement cannot resolve pair by pair, and the cluster step would
// then diagonalise most of the band on one thread.
namespace {

template <typename T>
struct LeArrays {
  T *A, *Y, *L, *d, *e, *e2, *lam, *vv, *pw, *bnd;
  int* cst;
};

// A, Y, L in `big` (3 n^2 values), the vectors in `vec` (8 n + 4 values, then n ints)
template <typename T>
LeArrays<T> le_arrays(T* big, T* vec, int n) {
  LeArrays<T> a;
  const size_t n2 = (size_t)n * n;
  a.A = big;
  a.Y = a.A + n2;
  a.L = a.Y + n2;
  a.d = vec;
  a.e = a.d + n;
  a.e2 = a.e + n;
  a.lam = a.e2 + n;
  a.vv = a.lam + n;
  a.pw = a.vv + n;
  a.bnd = a.pw + n;
  a.cst = reinterpret_cast<int*>(a.bnd + 4);
  return a;
}

template <typename T>
__device__ T le_block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T t = T(0);
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

template <typename T>
__global__ void k_le_init(const double* __restrict__ Ain, int n, T* __restrict__ A) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx % n), j = (int)(idx / n);
  A[idx] = (T)(0.5 * (Ain[i + (size_t)j * n] + Ain[j + (size_t)i * n]));
}

// One step k of the Householder reduction in two launches (a grid-wide result that is cheap
// to recompute is recomputed per CTA instead of taking a launch of its own):
//  part 1: every CTA forms the reflector v of column k in shared memory (the norm by a block
//  reduction that takes the same order in every CTA, so all CTAs hold the same v); CTA 0
//  publishes v (vv) and e[k]; warp i of the grid forms pw[i] = sum_j A[k+1+j, k+1+i] v[j].
//  Column k keeps x until part 2, because other CTAs still read it.
template <typename T>
__global__ void __launch_bounds__(256) k_le_house_matvec(const T* __restrict__ A, int n, int k,
                                                         T* __restrict__ vv, T* __restrict__ pw,
                                                         T* __restrict__ e) {
  extern __shared__ __align__(16) unsigned char le_sm[];
  T* vs = reinterpret_cast<T*>(le_sm);  // m values
  __shared__ T red[32];
  const int m = n - k - 1;
  const T* col = A + (k + 1) + (size_t)k * n;
  T xs = T(0);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const T c = col[i];
    vs[i] = c;
    xs += c * c;
  }
  const T xnorm = sqrt(le_block_sum(xs, red));
  const T x0 = col[0];
  const T alpha = (x0 >= T(0)) ? -xnorm : xnorm;
  const T vnorm2 = T(2) * (xnorm * xnorm - alpha * x0);
  const bool skip = !(vnorm2 > T(0));
  const T inv = skip ? T(0) : T(1) / sqrt(vnorm2);
  // each thread rewrites the entries it loaded
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    vs[i] = skip ? T(0) : (i == 0 ? vs[i] - alpha : vs[i]) * inv;
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) vv[i] = vs[i];
    if (threadIdx.x == 0) e[k] = skip ? x0 : alpha;
  }
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const T* c = A + (k + 1) + (size_t)(k + 1 + i) * n;
  T sum = T(0);
  for (int j = lane; j < m; j += 32) sum += c[j] * vs[j];
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) pw[i] = sum;
}

//  part 2: every CTA forms K = v . pw (same order in every CTA), then w = pw - K v on the fly
//  and the trailing block A -= 2 (v w^T + w v^T), four elements per thread; CTA 0 stores v in
//  column k below the diagonal (read by the back-transformation).
template <typename T>
__global__ void __launch_bounds__(256) k_le_w_update(T* __restrict__ A, int n, int k,
                                                     const T* __restrict__ vv,
                                                     const T* __restrict__ pw) {
  __shared__ T red[32];
  const int m = n - k - 1;
  T kp = T(0);
  for (int i = threadIdx.x; i < m; i += blockDim.x) kp += vv[i] * pw[i];
  const T K = le_block_sum(kp, red);
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < m; i += blockDim.x) A[(k + 1 + i) + (size_t)k * n] = vv[i];
  const long long mm = (long long)m * m;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const long long idx = ((long long)blockIdx.x * 4 + r) * blockDim.x + threadIdx.x;
    if (idx >= mm) break;
    const int i = (int)(idx % m), j = (int)(idx / m);
    const T wi = pw[i] - K * vv[i], wj = pw[j] - K * vv[j];
    A[(k + 1 + i) + (size_t)(k + 1 + j) * n] -= T(2) * (vv[i] * wj + wi * vv[j]);
  }
}

// d, e of the tridiagonal; e2 = e^2; Gershgorin bounds into bnd[0..1]
template <typename T>
__global__ void __launch_bounds__(1024) k_le_tridiag(const T* __restrict__ A, int n,
                                                     T* __restrict__ d, T* __restrict__ e,
                                                     T* __restrict__ e2, T* __restrict__ bnd) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = A[i + (size_t)i * n];
  __syncthreads();
  if (threadIdx.x == 0) {
    if (n >= 2) e[n - 2] = A[(n - 1) + (size_t)(n - 2) * n];
    e[n - 1] = T(0);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) e2[j] = (j < n - 1) ? e[j] * e[j] : T(0);
  if (threadIdx.x == 0) {
    T lo = d[0], hi = d[0];
    for (int j = 0; j < n; ++j) {
      const T r = (j > 0 ? fabs(e[j - 1]) : T(0)) + (j < n - 1 ? fabs(e[j]) : T(0));
      lo = fmin(lo, d[j] - r);
      hi = fmax(hi, d[j] + r);
    }
    bnd[0] = lo;
    bnd[1] = hi;
  }
}

// eigenvalue i by bisection on Sturm counts, its eigenvector of T by inverse iteration
// (column i of Y; L factors in column i of L), one thread per eigenvalue
// Eigenvalues of the tridiagonal (d, e) by multisection on Sturm counts, one warp per
// eigenvalue: each round the 32 lanes evaluate the count at 32 interior points of the bracket
// (33 equal parts) and a warp vote keeps the part that holds eigenvalue i, 33x per round where
// bisection gives 2x, so about 11 serial Sturm sweeps reach the FP64 resolution instead of
// about 55, and the warps of all eigenvalues spread over the GPU. Lane 0 then finds the
// eigenvector by inverse iteration with the LDL^T factors of T - lambda I (three passes from a
// start vector that differs per eigenvalue).
template <typename T>
__global__ void __launch_bounds__(256) k_le_multisect(int n, const T* __restrict__ d,
                                                      const T* __restrict__ e,
                                                      const T* __restrict__ e2,
                                                      const T* __restrict__ bnd,
                                                      T* __restrict__ lam, T* __restrict__ Y,
                                                      T* __restrict__ Ls) {
  const int i = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;  // whole warps leave together
  const T glo = bnd[0], ghi = bnd[1];
  const T tnorm = fmax(fabs(glo), fabs(ghi)) + T(1e-30);
  const T piv = EigEps<T>::v() * tnorm;
  T a = glo - piv, b = ghi + piv;  // count(a) <= i < count(b)
  for (int round = 0; round < 40; ++round) {
    const T x = a + (b - a) * (T)(lane + 1) * T(1.0 / 33.0);
    int cnt = 0;
    T q = d[0] - x;
    if (fabs(q) < piv) q = -piv;
    cnt += (q < T(0));
    for (int j = 1; j < n; ++j) {
      q = d[j] - x - e2[j - 1] / q;
      if (fabs(q) < piv) q = -piv;
      cnt += (q < T(0));
    }
    // the first interior point above eigenvalue i bounds it from above, the point before it
    // from below
    const unsigned above = __ballot_sync(0xffffffffu, cnt > i);
    const int k = above ? __ffs(above) - 1 : 32;
    const T xk = __shfl_sync(0xffffffffu, x, k < 32 ? k : 31);
    const T xl = __shfl_sync(0xffffffffu, x, k > 0 ? k - 1 : 0);
    const T na = (k == 0) ? a : xl;
    const T nb = (k == 32) ? b : xk;
    if (!(na > a || nb < b)) break;  // no interior point moved the bracket: resolution reached
    a = na;
    b = nb;
  }
  if (lane != 0) return;
  const T x = T(0.5) * (a + b);
  lam[i] = x;
  T* y = Y + (size_t)i * n;
  T* L = Ls + (size_t)i * n;
  for (int j = 0; j < n; ++j) {
    const unsigned hsh = (unsigned)(j + 1) * 2654435761u ^ (unsigned)(i + 1) * 40503u;
    y[j] = T(0.5) + (T)((hsh >> 8) & 0xffffu) * T(1.0 / 65536.0);
  }
  for (int rep = 0; rep < 3; ++rep) {
    T Dp = d[0] - x;
    if (fabs(Dp) < piv) Dp = piv;
    T zp = y[0];
    y[0] = zp / Dp;
    for (int j = 1; j < n; ++j) {
      const T l = e[j - 1] / Dp;
      L[j] = l;
      const T z = y[j] - l * zp;
      T Dj = d[j] - x - l * e[j - 1];
      if (fabs(Dj) < piv) Dj = piv;
      y[j] = z / Dj;
      zp = z;
      Dp = Dj;
    }
    for (int j = n - 2; j >= 0; --j) y[j] -= L[j + 1] * y[j + 1];
    T ss = T(0);
    for (int j = 0; j < n; ++j) ss += y[j] * y[j];
    const T sc = T(1) / sqrt(ss);
    for (int j = 0; j < n; ++j) y[j] *= sc;
  }
}

// clusters of eigenvalues closer than tol |T|: modified Gram-Schmidt, twice (one CTA)
template <typename T>
__global__ void __launch_bounds__(1024) k_le_clusters(int n, const T* __restrict__ lam,
                                                      const T* __restrict__ bnd, T tol,
                                                      T* __restrict__ Y,
                                                      int* __restrict__ cst) {
  __shared__ int kmax;
  const T tnorm = fmax(fabs(bnd[0]), fabs(bnd[1])) + T(1e-30);
  if (threadIdx.x == 0) {
    int start = 0, km = 0;
    for (int i = 0; i < n; ++i) {
      if (i > 0 && lam[i] - lam[i - 1] > tol * tnorm) start = i;
      cst[i] = start;
      km = max(km, i - start);
    }
    kmax = km;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 2; ++sweep)
    for (int pos = 1; pos <= kmax; ++pos) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (i - cst[i] != pos) continue;
        T* y = Y + (size_t)i * n;
        for (int jv = cst[i]; jv < i; ++jv) {
          const T* u = Y + (size_t)jv * n;
          T dot = T(0);
          for (int j = 0; j < n; ++j) dot += u[j] * y[j];
          for (int j = 0; j < n; ++j) y[j] -= dot * u[j];
        }
        T ss = T(0);
        for (int j = 0; j < n; ++j) ss += y[j] * y[j];
        const T sc = T(1) / sqrt(ss);
        for (int j = 0; j < n; ++j) y[j] *= sc;
      }
      __syncthreads();
    }
}

// The whole back-transformation Y <- H_0 H_1 ... H_{n-3} Y in one launch: columns are
// independent, so warp j applies every reflector to column j in turn: t = 2 v_k . y_j, then
// y_j -= t v_k, for k = n-3 down to 0
template <typename T>
__global__ void k_le_apply_all(const T* __restrict__ A, int n, T* __restrict__ Y) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  for (int k = n - 3; k >= 0; --k) {
    const int m = n - k - 1;
    const T* v = A + (k + 1) + (size_t)k * n;
    T* y = Y + (k + 1) + (size_t)j * n;
    T t = T(0);
    for (int i = lane; i < m; i += 32) t += v[i] * y[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    t *= T(2);
    for (int i = lane; i < m; i += 32) y[i] -= t * v[i];
    __syncwarp();  // the next reflector's rows are other lanes' rows of this one
  }
}

template <typename T>
__global__ void k_le_out(const T* __restrict__ Y, long long n2, double* __restrict__ V,
                         int* __restrict__ status) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n2) V[idx] = (double)Y[idx];
  if (idx == 0) status[0] = 1;
}

// FP64 tridiagonal solve on device-wide kernels: A, Y, L in `big` (3 n^2 doubles), vectors in
// `vec` (8 n + 4 doubles and n ints); V0 receives the eigenvectors (ascending eigenvalues)
cudaError_t le_stage(const double* Ain, int n, double* big, double* vec, double* V0, int* status,
                     cudaStream_t st) {
  using T = double;
  const LeArrays<T> a = le_arrays<T>(big, vec, n);
  const long long n2 = (long long)n * n;
  k_le_init<T><<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(Ain, n, a.A);
  const size_t vs_bytes = (size_t)n * sizeof(T);
  if (vs_bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_le_house_matvec<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vs_bytes);
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const long long mm = (long long)m * m;
    k_le_house_matvec<T><<<(m + 7) / 8, 256, (size_t)m * sizeof(T), st>>>(a.A, n, k, a.vv, a.pw,
                                                                          a.e);
    k_le_w_update<T><<<(unsigned)((mm + 1023) / 1024), 256, 0, st>>>(a.A, n, k, a.vv, a.pw);
  }
  k_le_tridiag<T><<<1, 1024, 0, st>>>(a.A, n, a.d, a.e, a.e2, a.bnd);
  k_le_multisect<T><<<(unsigned)(((long long)n * 32 + 255) / 256), 256, 0, st>>>(
      n, a.d, a.e, a.e2, a.bnd, a.lam, a.Y, a.L);
  k_le_clusters<T><<<1, 1024, 0, st>>>(n, a.lam, a.bnd, T(1e-10), a.Y, a.cst);
  k_le_apply_all<T><<<(n + 7) / 8, 256, 0, st>>>(a.A, n, a.Y);
  k_le_out<T><<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(a.Y, n2, V0, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sym_eig(const double* A, int n, double* theta, double* V, double* work,
                              int* status, cudaStream_t stream, void* oz, size_t oz_bytes,
                              int* oz_err) {
  const size_t n2 = (size_t)n * n;
  double* V0 = work;
  double* V1 = V0 + n2;
  double* P = V1 + n2;
  double* S = P + n2;
  double* G = S + n2;
  double* Ep = G + n2;
  double* lam = Ep + n2;          // n
  double* scal = lam + n;         // 4
  double* scratch = scal + 4;     // 2 n^2 + 2 n (final step)
  // threads of the one-CTA FP32 stage: 512 measured fastest at n = 80 (1.55 ms per Rayleigh-Ritz
  // dense part against 1.65 at 256, 1.90 at 128, 1.56 at 1024; the same Ritz values);
  // CS_EIG_THREADS (a multiple of 32, up to 1024) overrides
  int threads = 512;
  if (const char* et = getenv("CS_EIG_THREADS")) {
    const int v = atoi(et);
    if (v >= 32 && v <= 1024 && v % 32 == 0) threads = v;
  }
  // 1. FP32 eigendecomposition of sym(A) -> V0 (FP64 copy of the FP32 vectors)
  cudaError_t e;
  const size_t smem_b = (4 * n2 + 7 * (size_t)n) * sizeof(float);
  if (smem_b <= 200 * 1024) {
    // bisection + inverse iteration on the tridiagonal (parallel over eigenvalues)
    e = cudaFuncSetAttribute(k_sym_eig<float, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
    if (e != cudaSuccess) return e;
    k_sym_eig<float, true, true><<<1, threads, smem_b, stream>>>(A, n, nullptr, V0, nullptr,
                                                                 status);
  } else {
    // device-wide FP64 stage: A, Y, L in P, S, G; its vectors in Ep (free until the
    // refinement); status as the one-CTA solver's
    if ((e = le_stage(A, n, P, Ep, V0, status, stream)) != cudaSuccess) return e;
  }
  // 2. orthonormalise to FP64 precision (Newton-Schulz), then refine in FP64. The 25 n x n
  // products take the FP64 pipe (small_gemm) or, for large n when the caller hands over a
  // slice-product workspace, the exact slice products on the tensor cores: at n = 880 one
  // FP64-pipe product is about 1.1 ms at the pipe's peak
  const bool sliced = oz != nullptr && oz_err != nullptr && n > 256 &&
                      oz_gram_work_bytes(n, n, n, false) <= oz_bytes &&
                      oz_rotate_work_bytes(n, n, n) <= oz_bytes;
  // C = X^T Y (ta) or X Y, all n x n with leading dimension n
  auto prod = [&](bool ta, const double* X, const double* Y, double* C) -> cudaError_t {
    if (!sliced) return small_gemm(ta, X, Y, n, C, stream);
    return ta ? launch_oz_gram(X, n, Y, n, n, n, n, C, n, oz, oz_err, stream)
              : launch_oz_rotate(X, n, Y, n, n, n, n, C, n, oz, oz_err, stream);
  };
  // ||A||, the Ogita-Aishima bound and the Rayleigh quotients; grid-wide for large n (the
  // partial sums go to scratch, free until the final step)
  constexpr int kNormCtas = 304;
  auto oa_norms = [&](const double* Am, const double* Sm, const double* Gm, double* lm,
                      double* sc) {
    if (n > 256) {
      k_oa_norms_part<<<kNormCtas, 256, 0, stream>>>(Am, Sm, Gm, n, lm, scratch);
      k_oa_norms_fin<<<1, 32, 0, stream>>>(scratch, kNormCtas, sc);
    } else {
      k_oa_norms<<<1, 1024, 0, stream>>>(Am, Sm, Gm, n, lm, sc);
    }
  };
  double* Vc = V0;
  double* Vn = V1;
  for (int it = 0; it < 3; ++it) {
    if ((e = prod(true, Vc, Vc, G)) != cudaSuccess) return e;   // G = V^T V
    k_ns_factor<<<(unsigned)((n2 + 255) / 256), 256, 0, stream>>>(G, n, Ep);
    if ((e = prod(false, Vc, Ep, Vn)) != cudaSuccess) return e;
    std::swap(Vc, Vn);
  }
  for (int it = 0; it < 4; ++it) {
    if ((e = prod(false, A, Vc, P)) != cudaSuccess) return e;   // P = A V
    if ((e = prod(true, Vc, P, S)) != cudaSuccess) return e;    // S = V^T A V
    if ((e = prod(true, Vc, Vc, G)) != cudaSuccess) return e;   // G = V^T V
    oa_norms(A, S, G, lam, scal);
    k_oa_update<<<(unsigned)((n2 + 255) / 256), 256, 0, stream>>>(S, G, n, lam, scal, Ep);
    if ((e = prod(false, Vc, Ep, Vn)) != cudaSuccess) return e;  // V (I + E)
    std::swap(Vc, Vn);
  }
  if ((e = prod(false, A, Vc, P)) != cudaSuccess) return e;
  if ((e = prod(true, Vc, P, S)) != cudaSuccess) return e;
  if ((e = prod(true, Vc, Vc, G)) != cudaSuccess) return e;
  oa_norms(A, S, G, lam, scal);
  // 3. sort, clusters, output
  k_oa_final<<<1, 1024, 0, stream>>>(S, G, Vc, n, scal, theta, V, scratch, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ residual norms
__global__ void k_residuals(const double* __restrict__ X, long long ldx,
                            const double* __restrict__ HX, long long ldh, long long d,
                            const double* __restrict__ theta, double* __restrict__ resid) {
  const int col = blockIdx.x;
  const double th = theta[col];
  const double* x = X + (size_t)col * ldx;
  const double* hx = HX + (size_t)col * ldh;
  double s = 0.0;
  for (long long i = threadIdx.x; i < d; i += blockDim.x) {
    double r = hx[i] - th * x[i];
    s = fma(r, r, s);
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    resid[col] = sqrt(t);
  }
}

cudaError_t launch_residuals(const double* X, long long ldx, const double* HX, long long ldh,
                             long long d, int n, const double* theta, double* resid,
                             cudaStream_t stream) {
  k_residuals<<<n, 256, 0, stream>>>(X, ldx, HX, ldh, d, theta, resid);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ elementwise helpers
template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ x, long long ldx, B* __restrict__ y,
                          long long ldy, long long d, int n) {
  long long tot = d * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    long long j = e / d, i = e - j * d;
    y[i + j * ldy] = (B)x[i + j * ldx];
  }
}

static unsigned elem_grid(long long tot) {
  long long b = (tot + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_convert_f64_to_f32(const double* x, long long ldx, float* y, long long ldy,
                                      long long d, int n, cudaStream_t stream) {
  k_convert<double, float><<<elem_grid(d * n), 256, 0, stream>>>(x, ldx, y, ldy, d, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_f32_to_f64(const float* x, long long ldx, double* y, long long ldy,
                                      long long d, int n, cudaStream_t stream) {
  k_convert<float, double><<<elem_grid(d * n), 256, 0, stream>>>(x, ldx, y, ldy, d, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_copy_block(const T* x, long long ldx, T* y, long long ldy, long long d,
                              int n, cudaStream_t stream) {
  k_convert<T, T><<<elem_grid(d * n), 256, 0, stream>>>(x, ldx, y, ldy, d, n);
  return cudaGetLastError();
}
template cudaError_t launch_copy_block<double>(const double*, long long, double*, long long,
                                               long long, int, cudaStream_t);
template cudaError_t launch_copy_block<df64>(const df64*, long long, df64*, long long,
                                            long long, int, cudaStream_t);
template cudaError_t launch_copy_block<float>(const float*, long long, float*, long long,
                                              long long, int, cudaStream_t);

__global__ void k_scale_inv_sqrt(const double* __restrict__ x, double* __restrict__ y,
                                 long long d, const double* __restrict__ nrm2) {
  double s = rsqrt(nrm2[0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * s;
}

cudaError_t launch_scale_inv_sqrt(const double* x, double* y, long long d, const double* nrm2,
                                  cudaStream_t stream) {
  k_scale_inv_sqrt<<<elem_grid(d), 256, 0, stream>>>(x, y, d, nrm2);
  return cudaGetLastError();
}

__global__ void k_weighted_potential(const double* __restrict__ v, const double* __restrict__ wkj,
                                     long long tot, int n_phi, double* __restrict__ wv64,
                                     float* __restrict__ wv32, df64* __restrict__ wvdf) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    double w = wkj[e / n_phi] * v[e];
    wv64[e] = w;
    wv32[e] = (float)w;
    if (wvdf) wvdf[e] = df64(w);
  }
}

cudaError_t launch_weighted_potential(const double* v, const double* wkj, int n_kj, int n_phi,
                                      double* wv64, float* wv32, df64* wvdf,
                                      cudaStream_t stream) {
  long long tot = (long long)n_kj * n_phi;
  k_weighted_potential<<<elem_grid(tot), 256, 0, stream>>>(v, wkj, tot, n_phi, wv64, wv32, wvdf);
  return cudaGetLastError();
}

// double <-> double-float blocks (d x n, leading dimensions ldx / ldy); in place is allowed
// (same element size, each element read and written by one thread)
__global__ void k_to_df64(const double* x, long long ldx, df64* y, long long ldy, long long d,
                          int n) {
  const long long tot = d * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % d, j = e / d;
    y[i + j * ldy] = df64(x[i + j * ldx]);
  }
}
__global__ void k_from_df64(const df64* x, long long ldx, double* y, long long ldy, long long d,
                            int n) {
  const long long tot = d * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % d, j = e / d;
    y[i + j * ldy] = x[i + j * ldx].to_double();
  }
}
cudaError_t launch_to_df64(const double* x, long long ldx, df64* y, long long ldy, long long d,
                           int n, cudaStream_t stream) {
  k_to_df64<<<elem_grid(d * n), 256, 0, stream>>>(x, ldx, y, ldy, d, n);
  return cudaGetLastError();
}
cudaError_t launch_from_df64(const df64* x, long long ldx, double* y, long long ldy, long long d,
                             int n, cudaStream_t stream) {
  k_from_df64<<<elem_grid(d * n), 256, 0, stream>>>(x, ldx, y, ldy, d, n);
  return cudaGetLastError();
}

__global__ void k_build_tridiag(const double* __restrict__ al, const double* __restrict__ be2,
                                int k, double* __restrict__ T) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e % k, j = e / k;
    double v = 0.0;
    if (i == j) v = al[i];
    else if (i == j + 1) v = sqrt(be2[j]);
    else if (j == i + 1) v = sqrt(be2[i]);
    T[e] = v;
  }
}

cudaError_t launch_build_tridiag(const double* alpha, const double* beta2, int k, double* T,
                                 cudaStream_t stream) {
  k_build_tridiag<<<1, 256, 0, stream>>>(alpha, beta2, k, T);
  return cudaGetLastError();
}

}  // namespace cs
