// Device functions of the per-l radial GEMM tiles (internal), shared by the single-basis
// kernels (hx_kernels.cu) and the batched persistent kernel (batch.cu). Sec. 2.2.2 eqs. G_lmr
// and Arlm_to_coeff; one 64 x 64 output tile per call, 256 threads, 4 x 4 outputs each.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"
#include "hx_kernels.cuh"

namespace cs {

constexpr int RBM = 64, RBN = 64, RBK = 16;

__device__ __forceinline__ void locate_l_tile(int tile, int S, int& l, int& c0) {
  l = 0;
  for (;;) {
    int ct = ((2 * l + 1) * S + RBN - 1) / RBN;
    if (tile < ct) break;
    tile -= ct;
    ++l;
  }
  c0 = tile * RBN;
}

// G[k][l^2 + mi][s] = sum_n rad[l][k][n] X[(l^2 + mi) N + n + s ld],  column c = mi*S + s
template <typename T>
__device__ __forceinline__ void radial_synth_tile(const T* __restrict__ X, long long ld,
                                                  T* __restrict__ G, const T* __restrict__ rad,
                                                  int L, int N, int n_r, int S, int l, int c0,
                                                  int k0, T (*As)[RBM + 1], T (*Bs)[RBN + 1]) {
  const int ncol = (2 * l + 1) * S;
  const int L2 = L * L;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  MacAcc<T> acc[4][4];
  const T* radl = rad + (size_t)l * n_r * N;
  for (int n0 = 0; n0 < N; n0 += RBK) {
    for (int idx = tid; idx < RBM * RBK; idx += 256) {
      int nn = idx % RBK, kk = idx / RBK;
      int k = k0 + kk, n = n0 + nn;
      As[nn][kk] = (k < n_r && n < N) ? radl[(size_t)k * N + n] : T(0);
    }
    for (int idx = tid; idx < RBN * RBK; idx += 256) {
      int nn = idx % RBK, cc = idx / RBK;
      int c = c0 + cc, n = n0 + nn;
      T v = T(0);
      if (c < ncol && n < N) {
        int mi = c / S, s = c - mi * S;
        v = X[(size_t)(l * l + mi) * N + n + (size_t)s * ld];
      }
      Bs[nn][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RBK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j].add_prod(a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int k = k0 + ty + 16 * i;
    if (k >= n_r) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = c0 + tx + 16 * j;
      if (c < ncol) G[((size_t)k * L2 + l * l) * S + c] = acc[i][j].value();
    }
  }
}

// Z[alpha(l, mi, n), s] = sum_k rad[l][k][n] G[k][l^2 + mi][s], then the epilogue.
template <typename T>
__device__ __forceinline__ void radial_anal_tile(const T* __restrict__ G,
                                                 const T* __restrict__ rad, int L, int N,
                                                 int n_r, int S, const Epilogue<T>& ep, int l,
                                                 int c0, int nb0, T (*As)[RBM + 1],
                                                 T (*Bs)[RBN + 1]) {
  const int ncol = (2 * l + 1) * S;
  const int L2 = L * L;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // tx -> n, ty -> c
  MacAcc<T> acc[4][4];
  const T* radl = rad + (size_t)l * n_r * N;
  for (int k0 = 0; k0 < n_r; k0 += RBK) {
    for (int idx = tid; idx < RBM * RBK; idx += 256) {
      int nn = idx % RBM, kk = idx / RBM;
      int k = k0 + kk, n = nb0 + nn;
      As[kk][nn] = (k < n_r && n < N) ? radl[(size_t)k * N + n] : T(0);
    }
    for (int idx = tid; idx < RBN * RBK; idx += 256) {
      int cc = idx % RBN, kk = idx / RBN;
      int c = c0 + cc, k = k0 + kk;
      Bs[kk][cc] = (c < ncol && k < n_r) ? G[((size_t)k * L2 + l * l) * S + c] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RBK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j].add_prod(a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int c = c0 + ty + 16 * j;
    if (c >= ncol) continue;
    int mi = c / S, s = c - mi * S;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int n = nb0 + tx + 16 * i;
      if (n >= N) continue;
      size_t a = (size_t)(l * l + mi) * N + n;
      size_t o = a + (size_t)s * ep.ld_out;
      T z = acc[i][j].value();
      if (ep.mode == EP_PLAIN) {
        ep.out[o] = z;
        continue;
      }
      T x = ep.X[a + (size_t)s * ep.ld];
      T hx = ep.half_lambda[a] * x + z;
      if (ep.kb) hx += ep.kb[a + (size_t)s * ep.kb_ld];
      if (ep.src) hx += ep.src_w[s] * ep.src[a + (size_t)s * ep.src_ld];
      if (ep.mode == EP_APPLY) {
        ep.out[o] = hx;
      } else {  // EP_CHEB: out = cA (HX - c X) - cB Yprev   (out may alias Yprev)
        T y = ep.cA * (hx - ep.cshift * x);
        if (ep.Yprev) y -= ep.cB * ep.Yprev[o];
        ep.out[o] = y;
      }
    }
  }
}

}  // namespace cs
