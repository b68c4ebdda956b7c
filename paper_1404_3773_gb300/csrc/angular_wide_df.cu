// Angular block of H.X (Sec. 2.2.2 eq. Ar_lm, the inverse transform of Sec. 2.2.4) in
// double-float for large lmax, where the row-pair tile (one CTA per radial node and a few
// states, all harmonics in shared memory) no longer fits: three passes over a double-float
// intermediate FA in device memory, the same passes as the mixed precision's tensor-core block
// (angular_wide.cu) with register-tiled double-float products on the FP32 pipe:
//   L1  per mode m: E[t][s] = sum_{l - |m| even} Theta_lm(t) G[l,m][s], O likewise over odd
//       l - |m|, for the theta pairs t; FA(t) = E + O, FA(pi - t) = E - O.
//   P   per grid row (k, t): the four phi classes (cos / sin with m even / odd) summed at the
//       quarter angles q = 0 .. n_phi/4, the grid values at the four mirror angles as their
//       +- combinations times W V, folded back per class, and the quadrature per class; the
//       row's AP replaces its F.
//   L2  per mode m: G'[l,m][s] = sum_t Theta_lm(t) AP_par(t)[s], AP_par(t) = AP(t) +- AP(pi - t).
// States run in blocks of 32 (the three launches per block, one block-sized FA reused).
// Exact identities only: the result differs from the row-pair and row-stream kernels by
// rounding order.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "cs_internal.h"
#include "df64.cuh"
#include "hx_kernels.cuh"

namespace cs {

namespace {

constexpr int kDfSB = 32;  // states per block
constexpr int kDfThreads = 256;

__host__ __device__ inline int df_class_kap(int c, int i, int lmax) {
  const int m = (c == 0) ? 2 * i : (c == 2) ? 2 * i + 2 : 2 * i + 1;
  if (m > lmax) return -1;
  return c < 2 ? lmax + m : lmax - m;
}
__host__ __device__ inline int df_class_m(int c, int i) {
  return (c == 0) ? 2 * i : (c == 2) ? 2 * i + 2 : 2 * i + 1;
}

struct DfShape {
  int L, lmax, M2, Nt, NP, Np, Q, Qn, KL, KC;
};
__host__ __device__ inline DfShape df_shape(int L, int n_theta, int n_phi) {
  DfShape s;
  s.L = L;
  s.lmax = L - 1;
  s.M2 = 2 * L - 1;
  s.Nt = n_theta;
  s.NP = (n_theta + 1) / 2;
  s.Np = n_phi;
  s.Q = n_phi / 4;
  s.Qn = s.Q + 1;
  s.KL = (L + 1) / 2;          // l per parity, at most
  s.KC = s.lmax / 2 + 1;       // modes per phi class, at most
  return s;
}

// shared memory (df64 elements) of the three kernels
__host__ __device__ inline size_t df_l1_elems(const DfShape& s) {
  return (size_t)2 * s.NP * s.KL + (size_t)2 * s.KL * kDfSB;
}
__host__ __device__ inline size_t df_l2_elems(const DfShape& s) {
  return (size_t)2 * s.NP * s.KL + (size_t)2 * s.NP * kDfSB;
}
__host__ __device__ inline size_t df_p_elems(const DfShape& s) {
  return (size_t)4 * s.Qn * s.KC + (size_t)s.M2 * kDfSB + (size_t)4 * s.Qn * kDfSB + s.Np;
}

struct DfArgs {
  int L, n_r, Nt, Np, S, s0, nmr;
  const df64* theta;  // [pair t][packed (m, l)]
  const df64* trig;   // [cos | sin][m][q]
  const df64* wv;     // [k][t][p]
  df64* G;            // [k][lm][S]
  df64* FA;           // [k][t][kap][kDfSB] for this block
};

__device__ __forceinline__ int df_item_m(int it) {
  return it == 0 ? 0 : ((it & 1) ? (it + 1) / 2 : -(it / 2));
}

// Legendre rows of mode |m| = am for both parities: th[par][t][i] = Theta_{am+par+2i, am}(t)
__device__ __forceinline__ void df_load_theta(const DfArgs& a, const DfShape& sh, int am,
                                              df64* th) {
  const int rowlen = sh.L * (sh.L + 1) / 2, off = theta_off(sh.L, am);
  const int n = 2 * sh.NP * sh.KL;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int par = idx / (sh.NP * sh.KL), rem = idx - par * sh.NP * sh.KL;
    const int t = rem / sh.KL, i = rem - t * sh.KL;
    const int l = am + par + 2 * i;
    th[idx] = (l <= sh.lmax) ? a.theta[(size_t)t * rowlen + off + (l - am)] : df64(0.f, 0.f);
  }
}

// ------------------------------------------------------------------------------------ L1
__global__ void __launch_bounds__(kDfThreads) k_leg_synth_df(DfArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DfShape sh = df_shape(a.L, a.Nt, a.Np);
  const int L = sh.L, lmax = sh.lmax, L2 = L * L, M2 = sh.M2, NP = sh.NP, KL = sh.KL;
  const int Nt = a.Nt, S = a.S, ns = min(kDfSB, S - a.s0);
  const int r = blockIdx.x % a.nmr, k = blockIdx.x / a.nmr;
  const int it0 = (int)((long long)r * M2 / a.nmr), it1 = (int)((long long)(r + 1) * M2 / a.nmr);
  df64* th = reinterpret_cast<df64*>(smem_raw);   // [par][NP][KL]
  df64* gs = th + (size_t)2 * NP * KL;            // [par][KL][SB]
  df64* base = a.FA + (size_t)k * Nt * M2 * kDfSB;
  // tile: 2 pairs x 4 states, both parities
  const int ntile = ((NP + 1) / 2) * (kDfSB / 4);
  int cur_a = -1;
  for (int it = it0; it < it1; ++it) {
    const int m = df_item_m(it), am = m < 0 ? -m : m, kap = m + lmax;
    __syncthreads();  // the previous mode's reads are done
    if (am != cur_a) df_load_theta(a, sh, am, th);
    cur_a = am;
    for (int idx = threadIdx.x; idx < 2 * KL * kDfSB; idx += blockDim.x) {
      const int par = idx / (KL * kDfSB), rem = idx - par * KL * kDfSB;
      const int i = rem / kDfSB, s = rem - i * kDfSB;
      const int l = am + par + 2 * i;
      gs[idx] = (l <= lmax && s < ns) ? a.G[((size_t)k * L2 + l * l + l + m) * S + a.s0 + s]
                                      : df64(0.f, 0.f);
    }
    __syncthreads();
    for (int ti = threadIdx.x; ti < ntile; ti += blockDim.x) {
      const int t0 = 2 * (ti / (kDfSB / 4)), s0 = 4 * (ti % (kDfSB / 4));
      df64acc e[2][4], o[2][4];
      const int t1 = min(t0 + 1, NP - 1);
      const df64* te0 = th + (size_t)t0 * KL;
      const df64* te1 = th + (size_t)t1 * KL;
      const df64* to0 = te0 + (size_t)NP * KL;
      const df64* to1 = te1 + (size_t)NP * KL;
      for (int i = 0; i < KL; ++i) {
        const df64 ae[2] = {te0[i], te1[i]}, ao[2] = {to0[i], to1[i]};
        const float4* ge = reinterpret_cast<const float4*>(gs + (size_t)i * kDfSB + s0);
        const float4* go = reinterpret_cast<const float4*>(gs + (size_t)(KL + i) * kDfSB + s0);
        const float4 g0 = ge[0], g1 = ge[1], h0 = go[0], h1 = go[1];
        const df64 be[4] = {df64(g0.x, g0.y), df64(g0.z, g0.w), df64(g1.x, g1.y),
                            df64(g1.z, g1.w)};
        const df64 bo[4] = {df64(h0.x, h0.y), df64(h0.z, h0.w), df64(h1.x, h1.y),
                            df64(h1.z, h1.w)};
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            e[u][v].add_prod(ae[u], be[v]);
            o[u][v].add_prod(ao[u], bo[v]);
          }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int t = t0 + u;
        if (t >= NP) continue;
        const int tb = Nt - 1 - t;
        df64* ft = base + ((size_t)t * M2 + kap) * kDfSB + s0;
        df64* fb = base + ((size_t)tb * M2 + kap) * kDfSB + s0;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const df64 ev = e[u][v].value(), ov = o[u][v].value();
          ft[v] = ev + ov;
          if (tb != t) fb[v] = ev - ov;
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------- P
__global__ void __launch_bounds__(kDfThreads) k_phi_df(DfArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DfShape sh = df_shape(a.L, a.Nt, a.Np);
  const int lmax = sh.lmax, M2 = sh.M2, Qn = sh.Qn, Q = sh.Q, KC = sh.KC;
  const int Nt = a.Nt, Np = a.Np, L = sh.L;
  df64* tt = reinterpret_cast<df64*>(smem_raw);  // [c][q][i]
  df64* fs = tt + (size_t)4 * Qn * KC;           // [kap][SB]
  df64* hs = fs + (size_t)M2 * kDfSB;            // [c][q][SB]
  df64* ws = hs + (size_t)4 * Qn * kDfSB;        // [p]
  // class trig tables at the quarter angles, once per CTA
  for (int idx = threadIdx.x; idx < 4 * Qn * KC; idx += blockDim.x) {
    const int c = idx / (Qn * KC), rem = idx - c * Qn * KC;
    const int q = rem / KC, i = rem - q * KC;
    const int mm = df_class_m(c, i);
    df64 v(0.f, 0.f);
    if (mm <= lmax) v = a.trig[((size_t)(c < 2 ? 0 : L) + mm) * Qn + q];
    tt[idx] = v;
  }
  const long long ntiles = (long long)a.n_r * Nt;
  const int nsyn = ((Qn + 3) / 4) * (kDfSB / 2);   // synthesis tiles: 4 q x 2 states
  const int nana = 4 * ((KC + 3) / 4) * (kDfSB / 4);  // quadrature tiles: 4 modes x 4 states
  for (long long tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
    const int k = (int)(tl / Nt), t = (int)(tl % Nt);
    df64* frow = a.FA + (size_t)tl * M2 * kDfSB;
    const df64* wvr = a.wv + ((size_t)k * Nt + t) * Np;
    __syncthreads();  // the previous tile is done with fs, hs, ws (and tt is complete)
    {
      const float4* src = reinterpret_cast<const float4*>(frow);
      float4* dst = reinterpret_cast<float4*>(fs);
      for (int idx = threadIdx.x; idx < M2 * kDfSB / 2; idx += blockDim.x) dst[idx] = src[idx];
      for (int idx = threadIdx.x; idx < Np; idx += blockDim.x) ws[idx] = wvr[idx];
    }
    __syncthreads();
    // class sums at 4 quarter angles x 2 states, folded with W V into the four classes
    for (int ti = threadIdx.x; ti < nsyn; ti += blockDim.x) {
      const int q0 = 4 * (ti / (kDfSB / 2)), s0 = 2 * (ti % (kDfSB / 2));
      df64acc acc[4][4][2];
      int qq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) qq[u] = min(q0 + u, Qn - 1);
      for (int i = 0; i < KC; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int kap = df_class_kap(c, i, lmax);
          if (kap < 0) continue;
          const float4 f = *reinterpret_cast<const float4*>(fs + (size_t)kap * kDfSB + s0);
          const df64 fv[2] = {df64(f.x, f.y), df64(f.z, f.w)};
          const df64* tc = tt + (size_t)c * Qn * KC + i;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const df64 tv = tc[(size_t)qq[u] * KC];
            acc[c][u][0].add_prod(tv, fv[0]);
            acc[c][u][1].add_prod(tv, fv[1]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u;
        if (q >= Qn) continue;
        const df64 w1 = ws[q], w2 = ws[2 * Q - q], w3 = ws[(2 * Q + q) % Np],
                   w4 = ws[(4 * Q - q) % Np];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const df64 ce = acc[0][u][v].value(), co = acc[1][u][v].value();
          const df64 se = acc[2][u][v].value(), so = acc[3][u][v].value();
          const df64 cp = ce + co, cm = ce - co, sp = se + so, sm = se - so;
          const df64 zero(0.f, 0.f);
          const df64 g1 = w1 * (cp + sp);
          const df64 g2 = (q != Q) ? w2 * (cm - sm) : zero;
          const df64 g3 = (q != 0) ? w3 * (cm + sm) : zero;
          const df64 g4 = (q != 0 && q != Q) ? w4 * (cp - sp) : zero;
          const int s = s0 + v;
          hs[((size_t)0 * Qn + q) * kDfSB + s] = (g1 + g2) + (g3 + g4);
          hs[((size_t)1 * Qn + q) * kDfSB + s] = (g1 - g2) - (g3 - g4);
          hs[((size_t)2 * Qn + q) * kDfSB + s] = (g1 - g2) + (g3 - g4);
          hs[((size_t)3 * Qn + q) * kDfSB + s] = (g1 + g2) - (g3 + g4);
        }
      }
    }
    __syncthreads();
    // quadrature per class: AP[kap(c, i)][s] = sum_q T_c[q][i] h_c[q][s]
    for (int ti = threadIdx.x; ti < nana; ti += blockDim.x) {
      const int per_c = ((KC + 3) / 4) * (kDfSB / 4);
      const int c = ti / per_c, rem = ti - c * per_c;
      const int i0 = 4 * (rem / (kDfSB / 4)), s0 = 4 * (rem % (kDfSB / 4));
      int ii[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ii[u] = min(i0 + u, KC - 1);
      df64acc acc[4][4];
      const df64* tc = tt + (size_t)c * Qn * KC;
      const df64* hc = hs + (size_t)c * Qn * kDfSB + s0;
      for (int q = 0; q < Qn; ++q) {
        const df64* tq = tc + (size_t)q * KC;
        const df64 tv[4] = {tq[ii[0]], tq[ii[1]], tq[ii[2]], tq[ii[3]]};
        const float4* hp = reinterpret_cast<const float4*>(hc + (size_t)q * kDfSB);
        const float4 h0 = hp[0], h1 = hp[1];
        const df64 hv[4] = {df64(h0.x, h0.y), df64(h0.z, h0.w), df64(h1.x, h1.y),
                            df64(h1.z, h1.w)};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v].add_prod(tv[u], hv[v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        if (i >= KC) continue;
        const int kap = df_class_kap(c, i, lmax);
        if (kap < 0) continue;
        df64* dst = frow + (size_t)kap * kDfSB + s0;
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[v] = acc[u][v].value();
      }
    }
  }
}

// ------------------------------------------------------------------------------------ L2
__global__ void __launch_bounds__(kDfThreads) k_leg_anal_df(DfArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DfShape sh = df_shape(a.L, a.Nt, a.Np);
  const int L = sh.L, lmax = sh.lmax, L2 = L * L, M2 = sh.M2, NP = sh.NP, KL = sh.KL;
  const int Nt = a.Nt, S = a.S, ns = min(kDfSB, S - a.s0);
  const int r = blockIdx.x % a.nmr, k = blockIdx.x / a.nmr;
  const int it0 = (int)((long long)r * M2 / a.nmr), it1 = (int)((long long)(r + 1) * M2 / a.nmr);
  df64* th = reinterpret_cast<df64*>(smem_raw);   // [par][NP][KL]
  df64* ap = th + (size_t)2 * NP * KL;            // [par][NP][SB]
  const df64* base = a.FA + (size_t)k * Nt * M2 * kDfSB;
  const int per_par = ((KL + 1) / 2) * (kDfSB / 4);  // tiles: 2 l x 4 states per parity
  int cur_a = -1;
  for (int it = it0; it < it1; ++it) {
    const int m = df_item_m(it), am = m < 0 ? -m : m, kap = m + lmax;
    __syncthreads();
    if (am != cur_a) df_load_theta(a, sh, am, th);
    cur_a = am;
    // AP of the pair folded into even and odd parts (a self-mirror row enters the even part)
    for (int idx = threadIdx.x; idx < NP * kDfSB; idx += blockDim.x) {
      const int t = idx / kDfSB, s = idx - t * kDfSB, tb = Nt - 1 - t;
      const df64 x = base[((size_t)t * M2 + kap) * kDfSB + s];
      const df64 y = (tb != t) ? base[((size_t)tb * M2 + kap) * kDfSB + s] : df64(0.f, 0.f);
      ap[idx] = x + y;
      ap[(size_t)NP * kDfSB + idx] = (tb != t) ? x - y : df64(0.f, 0.f);
    }
    __syncthreads();
    for (int ti = threadIdx.x; ti < 2 * per_par; ti += blockDim.x) {
      const int par = ti / per_par, rem = ti - par * per_par;
      const int i0 = 2 * (rem / (kDfSB / 4)), s0 = 4 * (rem % (kDfSB / 4));
      const int i1 = min(i0 + 1, KL - 1);
      const df64* tp = th + (size_t)par * NP * KL;
      const df64* apb = ap + (size_t)par * NP * kDfSB + s0;
      df64acc acc[2][4];
      for (int t = 0; t < NP; ++t) {
        const df64 tv[2] = {tp[(size_t)t * KL + i0], tp[(size_t)t * KL + i1]};
        const float4* p = reinterpret_cast<const float4*>(apb + (size_t)t * kDfSB);
        const float4 h0 = p[0], h1 = p[1];
        const df64 hv[4] = {df64(h0.x, h0.y), df64(h0.z, h0.w), df64(h1.x, h1.y),
                            df64(h1.z, h1.w)};
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v].add_prod(tv[u], hv[v]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int l = am + par + 2 * (i0 + u);
        if (i0 + u >= KL || l > lmax) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (s0 + v < ns)
            a.G[((size_t)k * L2 + l * l + l + m) * S + a.s0 + s0 + v] = acc[u][v].value();
      }
    }
  }
}

}  // namespace

bool angular_wide_df_eligible(int L, int n_theta, int n_phi) {
  if (L < 1 || n_theta < 2 || n_phi < 8 || (n_phi & 3) != 0) return false;
  const DfShape s = df_shape(L, n_theta, n_phi);
  const size_t lim = 200 * 1024 / sizeof(df64);
  return df_l1_elems(s) <= lim && df_l2_elems(s) <= lim && df_p_elems(s) <= lim;
}

bool angular_wide_df_enabled(int L, int n_theta, int n_phi, int Q4) {
  if (!angular_wide_df_eligible(L, n_theta, n_phi)) return false;
  const char* e = getenv("CS_ANGULAR_KERNEL");
  if (e && e[0] == 'w') return true;
  if (e && e[0] != '\0') return false;
  return !angular_rp_fits<df64>(L, Q4);
}

size_t angular_wide_df_work_bytes(int L, int n_r, int n_theta) {
  return (size_t)n_r * n_theta * (2 * L - 1) * kDfSB * sizeof(df64);
}

cudaError_t launch_angular_wide_df(const AngArgs<df64>& a, df64* G, df64* FA,
                                   cudaStream_t stream) {
  if (!FA || !angular_wide_df_eligible(a.L, a.n_theta, a.n_phi) || a.S <= 0)
    return cudaErrorInvalidConfiguration;
  const DfShape s = df_shape(a.L, a.n_theta, a.n_phi);
  cudaError_t e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const size_t b1 = df_l1_elems(s) * sizeof(df64), b2 = df_l2_elems(s) * sizeof(df64);
  const size_t bp = df_p_elems(s) * sizeof(df64);
  if ((e = cudaFuncSetAttribute(k_leg_synth_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)b1)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_phi_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bp)) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_leg_anal_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)b2)) != cudaSuccess)
    return e;
  DfArgs w;
  w.L = a.L;
  w.n_r = a.n_r;
  w.Nt = a.n_theta;
  w.Np = a.n_phi;
  w.S = a.S;
  w.theta = a.theta;
  w.trig = a.trig;
  w.wv = a.wv;
  w.G = G;
  w.FA = FA;
  // Legendre passes: one CTA per (radial node, range of modes), about 4 CTAs per SM
  int nmr = (4 * nsm + a.n_r - 1) / a.n_r;
  if (nmr < 1) nmr = 1;
  if (nmr > s.M2) nmr = s.M2;
  w.nmr = nmr;
  int per_sm = (int)((228 * 1024) / (bp + 1024));
  if (per_sm < 1) per_sm = 1;
  long long pgrid = (long long)nsm * per_sm;
  const long long ptiles = (long long)a.n_r * a.n_theta;
  if (pgrid > ptiles) pgrid = ptiles;
  for (int s0 = 0; s0 < a.S; s0 += kDfSB) {
    w.s0 = s0;
    k_leg_synth_df<<<a.n_r * nmr, kDfThreads, b1, stream>>>(w);
    k_phi_df<<<(int)pgrid, kDfThreads, bp, stream>>>(w);
    k_leg_anal_df<<<a.n_r * nmr, kDfThreads, b2, stream>>>(w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cs
