// Dense FP64 pieces of the ChFSI iteration (Sec. 3.2.1): Gram matrices and block
// rotations for Cholesky-QR (Sec. 3.1.1: Cholesky after column scaling) and Rayleigh-
// Ritz, a one-CTA parallel cyclic Jacobi eigensolver for the projected matrix, residual
// norms, conversions and small vector helpers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

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

template <int U>
__global__ void __launch_bounds__(256) k_gram_partial(const double* __restrict__ A, long long lda,
                                                       const double* __restrict__ B,
                                                       long long ldb, long long d, int na,
                                                       int nb, long long rows,
                                                       double* __restrict__ partial) {
  constexpr int T = 16 * U;
  const int i0 = blockIdx.x * T, j0 = blockIdx.y * T;
  const int chunk = blockIdx.z;
  const long long r0 = (long long)chunk * rows;
  const long long r1 = min(d, r0 + rows);
  __shared__ double As[GK][T + 1];
  __shared__ double Bs[GK][T + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0.0;
  for (long long rb = r0; rb < r1; rb += GK) {
    for (int idx = tid; idx < GK * T; idx += 256) {
      int rr = idx % GK, cc = idx / GK;
      long long r = rb + rr;
      int i = i0 + cc, j = j0 + cc;
      As[rr][cc] = (r < r1 && i < na) ? A[r + (long long)i * lda] : 0.0;
      Bs[rr][cc] = (r < r1 && j < nb) ? B[r + (long long)j * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < GK; ++rr) {
      double a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = As[rr][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < U; ++v) b[v] = Bs[rr][ty + 16 * v];
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* P = partial + (size_t)chunk * na * nb;
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) {
      int i = i0 + tx + 16 * u, j = j0 + ty + 16 * v;
      if (i < na && j < nb) P[i + (size_t)j * na] = acc[u][v];
    }
}

// 32 elements x 8 chunk slices per 256-thread block; slices summed in a fixed order
__global__ void k_gram_reduce(const double* __restrict__ partial, int chunks, int na, int nb,
                              double* __restrict__ C, int ldc) {
  __shared__ double red[8][33];
  const int el = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + el;
  const int E = na * nb;
  double s = 0.0;
  if (e < E)
    for (int c = sl; c < chunks; c += 8) s += partial[(size_t)c * E + e];
  red[sl][el] = s;
  __syncthreads();
  if (sl == 0 && e < E) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += red[k][el];
    int i = e % na, j = e / na;
    C[i + (size_t)j * ldc] = t;
  }
}

cudaError_t launch_gram(const double* A, long long lda, const double* B, long long ldb,
                        long long d, int na, int nb, double* C, int ldc, double* partial,
                        cudaStream_t stream) {
  int u, ta, tb, chunks;
  long long rows;
  gram_shape(d, na, nb, u, ta, tb, chunks, rows);
  dim3 grid(ta, tb, chunks);
  switch (u) {
    case 1: k_gram_partial<1><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 2: k_gram_partial<2><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 3: k_gram_partial<3><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 4: k_gram_partial<4><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    case 5: k_gram_partial<5><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
    default: k_gram_partial<6><<<grid, 256, 0, stream>>>(A, lda, B, ldb, d, na, nb, rows, partial); break;
  }
  int tot = na * nb;
  k_gram_reduce<<<(tot + 31) / 32, 256, 0, stream>>>(partial, chunks, na, nb, C, ldc);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ C = alpha A Q + beta C
// 64 rows x (16U) columns per CTA; U from n so that 80 states are one column tile.
template <int U>
__global__ void __launch_bounds__(256) k_gemm_nn(const double* __restrict__ A, long long lda,
                                                  const double* __restrict__ Q, int ldq,
                                                  long long d, int K, int n, double alpha,
                                                  double beta, double* C, long long ldc) {
  constexpr int BM = 64, BN = 16 * U;
  const long long r0 = (long long)blockIdx.x * BM;
  const int j0 = blockIdx.y * BN;
  __shared__ double As[GK][BM + 1];  // As[k][r]
  __shared__ double Qs[GK][BN + 1];  // Qs[k][j]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][U];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0.0;
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int idx = tid; idx < GK * BM; idx += 256) {
      int rr = idx % BM, kk = idx / BM;
      long long r = r0 + rr;
      int k = k0 + kk;
      As[kk][rr] = (r < d && k < K) ? A[r + (long long)k * lda] : 0.0;
    }
    for (int idx = tid; idx < GK * BN; idx += 256) {
      int kk = idx % GK, jj = idx / GK;
      int k = k0 + kk, j = j0 + jj;
      Qs[kk][jj] = (k < K && j < n) ? Q[k + (long long)j * ldq] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[U];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < U; ++v) b[v] = Qs[kk][ty + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
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
      double* c = C + r + (long long)j * ldc;
      *c = (beta == 0.0) ? alpha * acc[u][v] : fma(alpha, acc[u][v], beta * *c);
    }
  }
}

cudaError_t launch_gemm_nn(const double* A, long long lda, const double* Q, int ldq,
                           long long d, int k, int n, double alpha, double beta, double* C,
                           long long ldc, cudaStream_t stream) {
  const int u = tile_u(n);
  dim3 grid((unsigned)((d + 63) / 64), (n + 16 * u - 1) / (16 * u));
  switch (u) {
    case 1: k_gemm_nn<1><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc); break;
    case 2: k_gemm_nn<2><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc); break;
    case 3: k_gemm_nn<3><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc); break;
    case 4: k_gemm_nn<4><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc); break;
    case 5: k_gemm_nn<5><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc); break;
    default: k_gemm_nn<6><<<grid, 256, 0, stream>>>(A, lda, Q, ldq, d, k, n, alpha, beta, C, ldc); break;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Cholesky-QR factor
// One CTA. Lc = work (n x n column-major, lower), Dv = work + n*n.
__global__ void __launch_bounds__(1024) k_cholqr_factor(const double* __restrict__ M, int n,
                                                         double* __restrict__ U,
                                                         double* __restrict__ work,
                                                         int* __restrict__ status) {
  double* Lc = work;
  double* Dv = work + (size_t)n * n;
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
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
  // right-looking Cholesky, lower triangle of Lc
  for (int j = 0; j < n; ++j) {
    __shared__ double ljj;
    if (tid == 0) {
      double p = Lc[j + (size_t)j * n];
      if (!(p > 0.0) || !isfinite(p)) {
        fail = j + 1;
        ljj = 1.0;
      } else {
        ljj = sqrt(p);
      }
      Lc[j + (size_t)j * n] = ljj;
    }
    __syncthreads();
    if (fail) {
      if (tid == 0) status[0] = fail;
      return;
    }
    for (int i = j + 1 + tid; i < n; i += nt) Lc[i + (size_t)j * n] /= ljj;
    __syncthreads();
    const int rem = n - j - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      int i = j + 1 + e % rem, k = j + 1 + e / rem;
      if (i >= k) Lc[i + (size_t)k * n] -= Lc[i + (size_t)j * n] * Lc[k + (size_t)j * n];
    }
    __syncthreads();
  }
  // U = D R^{-1} = D (L^{-1})^T : column c of L^{-1} by forward substitution (thread per c)
  for (int c = tid; c < n; c += nt) {
    for (int i = 0; i < n; ++i) U[i + (size_t)c * n] = 0.0;
  }
  __syncthreads();
  for (int c = tid; c < n; c += nt) {
    // y = L^{-1} e_c, y_i = 0 for i < c; store y_i into U[c][i] (row c of U^T = col c ...)
    for (int i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= Lc[i + (size_t)k * n] * U[c + (size_t)k * n];
      U[c + (size_t)i * n] = s / Lc[i + (size_t)i * n];
    }
  }
  __syncthreads();
  // U currently holds (L^{-1})^T (upper): U[c][i] = (L^{-1})[i][c]; scale rows by D
  for (int e = tid; e < n * n; e += nt) {
    int i = e % n;
    U[e] *= Dv[i];
  }
  if (tid == 0) status[0] = 0;
}

cudaError_t launch_cholqr_factor(const double* M, int n, double* U, double* work, int* status,
                                 cudaStream_t stream) {
  k_cholqr_factor<<<1, 1024, 0, stream>>>(M, n, U, work, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ parallel Jacobi
// Cyclic Jacobi with round-robin (tournament) ordering: in each round n/2 disjoint pairs
// (p, q) rotate at once; n-1 rounds form a sweep. The rotation zeroing A_pq is the
// classical symmetric Schur rotation (t = sign(tau)/(|tau| + sqrt(1 + tau^2))); the
// annihilated pair is then set to zero exactly. A pair is rotated only if
// |A_pq| > 1e-15 ||A||_F (below that the eigenvalues move by O(1e-30 ||A||^2 / gap)); the
// iteration stops after a sweep without rotations (at most 50 sweeps). Round r of the
// tournament pairs position i with position np-1-i, where position 0 holds player 0 and
// position p >= 1 holds player 1 + (p - 1 + r) mod (np - 1).
// One CTA; A (n x n) in work, V output. Odd n is padded by one dummy index.
template <bool SMEM>
__global__ void __launch_bounds__(1024) k_jacobi(const double* __restrict__ Ain, int n,
                                                  double* __restrict__ theta,
                                                  double* __restrict__ Vout,
                                                  double* __restrict__ work,
                                                  int* __restrict__ status) {
  extern __shared__ double sh[];
  const int np = (n + 1) & ~1;  // even player count
  const int half = np / 2;
  int* pp = reinterpret_cast<int*>(sh) + np;  // [half] (first np ints unused)
  int* qq = pp + half;                     // [half]
  double* cs = reinterpret_cast<double*>(qq + half);  // [half]; 2*np ints = 8-byte aligned
  double* sn = cs + half;                             // [half]
  __shared__ double red[32];
  __shared__ int rotations;
  __shared__ double floor_abs;
  // working copies: in shared memory when they fit (n <= 112), else in global memory
  double* A = SMEM ? sn + half : work;
  double* V = SMEM ? sn + half + (size_t)n * n : Vout;
  const int tid = threadIdx.x, nt = blockDim.x;
  double fro = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    int i = e % n, j = e / n;
    double a = 0.5 * (Ain[i + (size_t)j * n] + Ain[j + (size_t)i * n]);
    A[e] = a;
    V[e] = (i == j) ? 1.0 : 0.0;
    fro += a * a;
  }
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if ((tid & 31) == 0) red[tid >> 5] = fro;
  __syncthreads();
  if (tid == 0) {
    double f = 0.0;
    for (int w = 0; w < (nt + 31) / 32; ++w) f += red[w];
    floor_abs = 1e-300 + 1e-15 * sqrt(f);
  }
  __syncthreads();
  int sweep = 0;
  bool converged = false;
  const int max_sweeps = 50;
  for (sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotations = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      // pairs from the current positions: (pos[i], pos[np-1-i])
      for (int i = tid; i < half; i += nt) {
        const int pa = i, pb = np - 1 - i;
        int a = (pa == 0) ? 0 : 1 + (pa - 1 + round) % (np - 1);
        int b = 1 + (pb - 1 + round) % (np - 1);
        int p = min(a, b), q = max(a, b);
        double c = 1.0, s = 0.0;
        if (q < n) {
          double apq = A[p + (size_t)q * n];
          double app = A[p + (size_t)p * n], aqq = A[q + (size_t)q * n];
          if (fabs(apq) > floor_abs) {
            double tau = (aqq - app) / (2.0 * apq);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = rsqrt(1.0 + t * t);
            s = t * c;
            atomicAdd(&rotations, 1);
          } else {
            q = n;  // no rotation for this pair
          }
        }
        pp[i] = p;
        qq[i] = q;
        cs[i] = c;
        sn[i] = s;
      }
      __syncthreads();
      // rows: A <- J^T A  (rows p, q of every column)
      for (int e = tid; e < half * n; e += nt) {
        int i = e % half, col = e / half;
        int p = pp[i], q = qq[i];
        if (q >= n) continue;
        double c = cs[i], s = sn[i];
        double ap = A[p + (size_t)col * n], aq = A[q + (size_t)col * n];
        A[p + (size_t)col * n] = c * ap - s * aq;
        A[q + (size_t)col * n] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J and V <- V J
      for (int e = tid; e < half * n; e += nt) {
        int i = e % half, row = e / half;
        int p = pp[i], q = qq[i];
        if (q >= n) continue;
        double c = cs[i], s = sn[i];
        double ap = A[row + (size_t)p * n], aq = A[row + (size_t)q * n];
        A[row + (size_t)p * n] = c * ap - s * aq;
        A[row + (size_t)q * n] = s * ap + c * aq;
        double vp = V[row + (size_t)p * n], vq = V[row + (size_t)q * n];
        V[row + (size_t)p * n] = c * vp - s * vq;
        V[row + (size_t)q * n] = s * vp + c * vq;
      }
      __syncthreads();
      // the rotation annihilates A_pq; remove its rounding residue
      for (int i = tid; i < half; i += nt) {
        int p = pp[i], q = qq[i];
        if (q < n) {
          A[p + (size_t)q * n] = 0.0;
          A[q + (size_t)p * n] = 0.0;
        }
      }
      __syncthreads();
    }
    if (rotations == 0) {
      converged = true;
      break;
    }
    __syncthreads();
  }
  // sort ascending: rank of each diagonal entry (ties by index), permute V columns
  double* tmpv = work + (size_t)n * n;  // n diagonal values
  for (int i = tid; i < n; i += nt) tmpv[i] = A[i + (size_t)i * n];
  __syncthreads();
  double* Vtmp = SMEM ? Vout : A;  // A is free once its diagonal is saved
  for (int i = tid; i < n; i += nt) {
    double vi = tmpv[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double vj = tmpv[j];
      rank += (vj < vi) || (vj == vi && j < i);
    }
    theta[rank] = vi;
    for (int r = 0; r < n; ++r) Vtmp[r + (size_t)rank * n] = V[r + (size_t)i * n];
  }
  __syncthreads();
  if (!SMEM)
    for (int e = tid; e < n * n; e += nt) Vout[e] = A[e];
  if (tid == 0) status[0] = converged ? sweep + 1 : -(sweep + 1);
}

cudaError_t launch_jacobi_eig(const double* A, int n, double* theta, double* V, double* work,
                              int* status, cudaStream_t stream) {
  int np = (n + 1) & ~1;
  int half = np / 2;
  size_t smem = (size_t)(np + 2 * half) * sizeof(int) + 2 * half * sizeof(double) + 16;  // pp, qq, cs, sn
  int threads = n <= 64 ? 256 : 1024;
  size_t smem_full = smem + 2 * (size_t)n * n * sizeof(double);
  if (smem_full <= 200 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_jacobi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_full);
    if (e != cudaSuccess) return e;
    k_jacobi<true><<<1, threads, smem_full, stream>>>(A, n, theta, V, work, status);
  } else {
    k_jacobi<false><<<1, threads, smem, stream>>>(A, n, theta, V, work, status);
  }
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
                                     float* __restrict__ wv32) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    double w = wkj[e / n_phi] * v[e];
    wv64[e] = w;
    wv32[e] = (float)w;
  }
}

cudaError_t launch_weighted_potential(const double* v, const double* wkj, int n_kj, int n_phi,
                                      double* wv64, float* wv32, cudaStream_t stream) {
  long long tot = (long long)n_kj * n_phi;
  k_weighted_potential<<<elem_grid(tot), 256, 0, stream>>>(v, wkj, tot, n_phi, wv64, wv32);
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
