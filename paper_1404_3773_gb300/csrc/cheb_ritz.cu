// Residual form of the Chebyshev filter (Sec. 3.2.1) for a block of Ritz vectors (internal).
//
// For Ritz vectors X with Ritz values Theta and residual block R = H X - X Theta, the scaled
// filter Y_m = p_m(H) X splits into an exact part and a deviation:
//   Y_i = X s_i(Theta) + D_i,   s_i = the same scaled polynomial on the scalars theta_j,
//   D_0 = 0,  D_1 = (sigma_1 / e) R,
//   D_{i+1} = (2 sigma_{i+1} / e) [(H - c) D_i + s_i(Theta) R] - sigma_i sigma_{i+1} D_{i-1}.
// (Subtract X s_{i+1}(Theta) from the recurrence of Y_{i+1} and use (H - c) X = X (Theta - c)
// + R.) In exact arithmetic Y_m is the plain filter's result for any Theta; in floating point
// the H products act only on D, whose size follows the residual, so the rounding error of a
// reduced-precision H.X scales with ||R|| instead of ||X||. The kernels here form the weights
// s_i(theta_j), R and D_1, and the final X s_m(Theta) + D_m; the recurrence itself is the
// radial-analysis epilogue (its src term).
#include <cuda_runtime.h>

#include "df64.cuh"
#include "hx_kernels.cuh"

namespace cs {

namespace {

__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(df64 x) { return x.to_double(); }
template <typename T>
__device__ __forceinline__ T from_d(double x) { return T(x); }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return (float)x; }

// wd[i * n + j] = s_i(theta_j) for i = 0 .. m (FP64), wt = the same rounded to T
template <typename T>
__global__ void k_cheb_weights(const double* __restrict__ theta, int n, int m, double c,
                               double e, double s1, double* __restrict__ wd, T* __restrict__ wt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double x = theta[j] - c;
  double sp = 1.0, sc = (s1 / e) * x, sig = s1;
  wd[j] = 1.0;
  wt[j] = from_d<T>(1.0);
  if (m >= 1) {
    wd[n + j] = sc;
    wt[n + j] = from_d<T>(sc);
  }
  for (int i = 1; i < m; ++i) {
    const double sn = 1.0 / (2.0 / s1 - sig);
    const double nx = (2.0 * sn / e) * x * sc - sig * sn * sp;
    sp = sc;
    sc = nx;
    sig = sn;
    wd[(size_t)(i + 1) * n + j] = sc;
    wt[(size_t)(i + 1) * n + j] = from_d<T>(sc);
  }
}

// R = H X - X Theta (rounded to T) and D_1 = (sigma_1 / e) R (rounded to T), d x n blocks
template <typename T>
__global__ void k_ritz_residual(const double* __restrict__ X, long long ldx,
                                const double* __restrict__ HX, long long ldh,
                                const double* __restrict__ theta, long long d, double f1,
                                T* __restrict__ R, T* __restrict__ D1) {
  const int s = blockIdx.y;
  const double th = theta[s];
  const double* x = X + (size_t)s * ldx;
  const double* hx = HX + (size_t)s * ldh;
  T* r = R + (size_t)s * d;
  T* d1 = D1 + (size_t)s * d;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < d;
       a += (long long)gridDim.x * blockDim.x) {
    const double v = fma(-th, x[a], hx[a]);
    r[a] = from_d<T>(v);
    d1[a] = from_d<T>(f1 * v);
  }
}

// X <- X s_m(Theta) + D_m
template <typename T>
__global__ void k_ritz_combine(double* __restrict__ X, long long ldx, const T* __restrict__ D,
                               long long d, const double* __restrict__ sm) {
  const int s = blockIdx.y;
  const double w = sm[s];
  double* x = X + (size_t)s * ldx;
  const T* dm = D + (size_t)s * d;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < d;
       a += (long long)gridDim.x * blockDim.x)
    x[a] = fma(w, x[a], to_d(dm[a]));
}

int row_blocks(long long d) {
  long long b = (d + 255) / 256;
  return (int)(b < 64 ? b : 64);
}

}  // namespace

template <typename T>
cudaError_t launch_cheb_weights(const double* theta, int n, int m, double c, double e, double s1,
                                double* wd, T* wt, cudaStream_t stream) {
  k_cheb_weights<T><<<(n + 127) / 128, 128, 0, stream>>>(theta, n, m, c, e, s1, wd, wt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ritz_residual(const double* X, long long ldx, const double* HX, long long ldh,
                                 const double* theta, long long d, int n, double f1, T* R, T* D1,
                                 cudaStream_t stream) {
  dim3 grid(row_blocks(d), n);
  k_ritz_residual<T><<<grid, 256, 0, stream>>>(X, ldx, HX, ldh, theta, d, f1, R, D1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ritz_combine(double* X, long long ldx, const T* D, long long d, int n,
                                const double* sm, cudaStream_t stream) {
  dim3 grid(row_blocks(d), n);
  k_ritz_combine<T><<<grid, 256, 0, stream>>>(X, ldx, D, d, sm);
  return cudaGetLastError();
}

#define CS_RITZ_INST(T)                                                                       \
  template cudaError_t launch_cheb_weights<T>(const double*, int, int, double, double, double, \
                                              double*, T*, cudaStream_t);                      \
  template cudaError_t launch_ritz_residual<T>(const double*, long long, const double*,        \
                                               long long, const double*, long long, int,       \
                                               double, T*, T*, cudaStream_t);                  \
  template cudaError_t launch_ritz_combine<T>(double*, long long, const T*, long long, int,    \
                                              const double*, cudaStream_t);
CS_RITZ_INST(double)
CS_RITZ_INST(float)
CS_RITZ_INST(df64)
#undef CS_RITZ_INST

}  // namespace cs
