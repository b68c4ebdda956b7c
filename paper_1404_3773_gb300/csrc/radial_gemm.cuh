// Register-blocked FP32 tiles of the per-l radial contractions of H.X (internal), Sec. 2.2.2
// eqs. G_lmr (synthesis) and Arlm_to_coeff (analysis, with the epilogue of hx_device.cuh):
//   synthesis : G[k][l^2 + mi][s]   = sum_n R_ln(r_k) X[(l^2 + mi) N + n + s ld]   (M = n_r, K = N)
//   analysis  : Z[(l^2 + mi) N + n, s] = sum_k R_ln(r_k) G[k][l^2 + mi][s]         (M = N, K = n_r)
// with column c = mi S + s of the l block. A CTA computes a (16 RM) x 128 output tile with 256
// threads, RM x 8 outputs each; every k step costs RM + 2 shared loads (RM of them broadcasts in
// the synthesis) for 8 RM FMAs. The thread layout follows the output's memory order so that the
// stores coalesce: in the synthesis (rows of G contiguous in the column) a thread holds rows
// RM ty .. RM ty + RM - 1 and columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3; in the
// analysis (output column-major, rows contiguous) it holds rows tr + 16 i and columns
// 8 tc .. 8 tc + 7. K runs in chunks of 16; the next chunk's global loads are issued into
// registers before the current chunk's FMAs (double-buffered shared memory, one barrier per
// chunk). The B tile's rows are padded to 132 floats so that its staging stores spread over
// the banks.
#pragma once

#include <cuda_runtime.h>

#include "hx_device.cuh"
#include "hx_kernels.cuh"

namespace cs {

constexpr int kRgBN = 128, kRgBK = 16, kRgThreads = 256;

__host__ __device__ inline int rg_col_tiles_l(int l, int S) {
  return ((2 * l + 1) * S + kRgBN - 1) / kRgBN;
}

__device__ __forceinline__ void rg_locate(int tile, int S, int& l, int& c0) {
  l = 0;
  for (;;) {
    const int ct = rg_col_tiles_l(l, S);
    if (tile < ct) break;
    tile -= ct;
    ++l;
  }
  c0 = tile * kRgBN;
}

constexpr int kRgBNp = kRgBN + 4;  // padded B-tile row

// rows per thread for a contraction with M output rows (tile = 16 RM rows)
__host__ __device__ inline int rg_rm(int M) {
  const int rm = (M + 15) / 16;
  return rm < 1 ? 1 : (rm > 8 ? 8 : rm);
}

__host__ __device__ inline int rg_col_tiles(int L, int S) {
  int t = 0;
  for (int l = 0; l < L; ++l) t += rg_col_tiles_l(l, S);
  return t;
}

// shared memory of one tile: two buffers of A (BK x BM) and B (BK x BNp) floats
template <int RM>
__host__ __device__ constexpr int rg_smem_floats() {
  return 2 * kRgBK * (16 * RM) + 2 * kRgBK * kRgBNp;
}

// MODE 0: synthesis (A = R_l [k][n], B gathered from X, output rows to G)
// MODE 1: analysis (A = R_l^T, B = G rows, output through the epilogue)
template <int MODE, int RM>
__device__ __forceinline__ void radial_gemm_tile(const float* __restrict__ X, long long ldx,
                                                 float* __restrict__ G,
                                                 const float* __restrict__ rad, int L, int N,
                                                 int n_r, int S, const Epilogue<float>& ep,
                                                 int l, int c0, int m0, float* smem) {
  constexpr int BM = 16 * RM, BN = kRgBN, BNp = kRgBNp, BK = kRgBK;
  constexpr int AE = BK * BM / kRgThreads;  // A elements staged per thread (BM <= 256)
  constexpr int BE = BK * BN / kRgThreads;  // B elements staged per thread (8)
  const int M = (MODE == 0) ? n_r : N;
  const int K = (MODE == 0) ? N : n_r;
  const int ncol = (2 * l + 1) * S;
  const int L2 = L * L;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float* As = smem;                 // [2][BK][BM]
  float* Bs = smem + 2 * BK * BM;   // [2][BK][BNp]
  const float* radl = rad + (size_t)l * n_r * N;

  float ra[AE > 0 ? AE : 1], rb[BE];
  // staging of chunk k0 into registers
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < AE; ++u) {
      const int e = tid + u * kRgThreads;   // e over (kk, m), m fastest
      const int kk = e / BM, mm = e - kk * BM;
      const int k = k0 + kk, m = m0 + mm;
      float v = 0.f;
      if (k < K && m < M) v = (MODE == 0) ? radl[(size_t)m * N + k] : radl[(size_t)k * N + m];
      ra[u] = v;
    }
#pragma unroll
    for (int u = 0; u < BE; ++u) {
      const int e = tid + u * kRgThreads;
      int kk, cc;
      if (MODE == 0) {   // X gather: consecutive threads along k (contiguous in X)
        kk = e % BK;
        cc = e / BK;
      } else {           // G rows: consecutive threads along columns (contiguous in G)
        cc = e % BN;
        kk = e / BN;
      }
      const int k = k0 + kk, c = c0 + cc;
      float v = 0.f;
      if (k < K && c < ncol) {
        if (MODE == 0) {
          const int mi = c / S, s = c - mi * S;
          v = X[(size_t)(l * l + mi) * N + k + (size_t)s * ldx];
        } else {
          v = G[((size_t)k * L2 + l * l) * S + c];
        }
      }
      rb[u] = v;
    }
  };
  auto stash = [&](int buf) {
    float* a = As + buf * BK * BM;
    float* b = Bs + buf * BK * BNp;
#pragma unroll
    for (int u = 0; u < AE; ++u) a[tid + u * kRgThreads] = ra[u];
#pragma unroll
    for (int u = 0; u < BE; ++u) {
      const int e = tid + u * kRgThreads;
      int kk, cc;
      if (MODE == 0) {
        kk = e % BK;
        cc = e / BK;
      } else {
        cc = e % BN;
        kk = e / BN;
      }
      b[kk * BNp + cc] = rb[u];
    }
  };

  float acc[RM][8];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int nchunk = (K + BK - 1) / BK;
  fetch(0);
  stash(0);
  __syncthreads();
  for (int ch = 0; ch < nchunk; ++ch) {
    const int buf = ch & 1;
    if (ch + 1 < nchunk) fetch((ch + 1) * BK);
    const float* a = As + buf * BK * BM;
    const float* b = Bs + buf * BK * BNp;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float av[RM], bv[8];
      if (MODE == 0) {
#pragma unroll
        for (int i = 0; i < RM; ++i) av[i] = a[kk * BM + RM * ty + i];
        const float4 b0 = *reinterpret_cast<const float4*>(b + kk * BNp + 4 * tx);
        const float4 b1 = *reinterpret_cast<const float4*>(b + kk * BNp + 64 + 4 * tx);
        bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
        bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
      } else {
#pragma unroll
        for (int i = 0; i < RM; ++i) av[i] = a[kk * BM + tx + 16 * i];
        const float4 b0 = *reinterpret_cast<const float4*>(b + kk * BNp + 8 * ty);
        const float4 b1 = *reinterpret_cast<const float4*>(b + kk * BNp + 8 * ty + 4);
        bv[0] = b0.x; bv[1] = b0.y; bv[2] = b0.z; bv[3] = b0.w;
        bv[4] = b1.x; bv[5] = b1.y; bv[6] = b1.z; bv[7] = b1.w;
      }
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (ch + 1 < nchunk) stash(buf ^ 1);
    __syncthreads();
  }

  // outputs
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const int m = m0 + ((MODE == 0) ? RM * ty + i : tx + 16 * i);
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = c0 + ((MODE == 0) ? ((j < 4) ? 4 * tx + j : 64 + 4 * tx + (j - 4)) : 8 * ty + j);
      if (c >= ncol) continue;
      if (MODE == 0) {
        G[((size_t)m * L2 + l * l) * S + c] = acc[i][j];
      } else {
        const int mi = c / S, s = c - mi * S;
        const size_t a_ = (size_t)(l * l + mi) * N + m;
        const size_t o = a_ + (size_t)s * ep.ld_out;
        const float z = acc[i][j];
        if (ep.mode == EP_PLAIN) {
          ep.out[o] = z;
          continue;
        }
        // every rounding is spelled out (fmaf, __fmul_rn, __fadd_rn), so the compiler cannot
        // contract differently from one kernel that embeds this tile to another: the batched
        // forms stay bitwise equal to the single-cluster launches
        const float x = ep.X[a_ + (size_t)s * ep.ld];
        float hx = fmaf(ep.half_lambda[a_], x, z);
        if (ep.kb) hx = __fadd_rn(hx, ep.kb[a_ + (size_t)s * ep.kb_ld]);
        if (ep.src) hx = fmaf(ep.src_w[s], ep.src[a_ + (size_t)s * ep.src_ld], hx);
        if (ep.mode == EP_APPLY) {
          ep.out[o] = hx;
        } else {  // EP_CHEB: out = cA (HX - c X) - cB Yprev   (out may alias Yprev)
          float y = __fmul_rn(ep.cA, fmaf(-ep.cshift, x, hx));
          if (ep.Yprev) y = fmaf(-ep.cB, ep.Yprev[o], y);
          ep.out[o] = y;
        }
      }
    }
  }
}

// runtime choice of RM (1 .. 8) for a tile of the given mode
template <int MODE>
__device__ __forceinline__ void radial_gemm_tile_rm(int rm, const float* __restrict__ X,
                                                    long long ldx, float* __restrict__ G,
                                                    const float* __restrict__ rad, int L, int N,
                                                    int n_r, int S, const Epilogue<float>& ep,
                                                    int l, int c0, int m0, float* smem) {
  switch (rm) {
    case 1: radial_gemm_tile<MODE, 1>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
    case 2: radial_gemm_tile<MODE, 2>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
    case 3: radial_gemm_tile<MODE, 3>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
    case 4: radial_gemm_tile<MODE, 4>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
    case 5: radial_gemm_tile<MODE, 5>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
    case 6: radial_gemm_tile<MODE, 6>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
    case 7: radial_gemm_tile<MODE, 7>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
    default: radial_gemm_tile<MODE, 8>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, m0, smem); break;
  }
}

}  // namespace cs
