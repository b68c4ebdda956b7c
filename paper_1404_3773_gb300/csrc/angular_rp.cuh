// Device function of the row-pair angular block (internal), shared by the single-basis kernel
// (angular_rp.cu) and the batched persistent kernel (batch.cu). See angular_rp.cu.
#pragma once

#include <cuda_runtime.h>

#include "cs_internal.h"
#include "df64.cuh"
#include "hx_kernels.cuh"

namespace cs {

template <typename T, int ST>
struct Vec;
template <>
struct Vec<float, 8> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    float4 a = reinterpret_cast<const float4*>(p)[0];
    float4 b = reinterpret_cast<const float4*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static __device__ __forceinline__ void store(float* p, const float* v) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
};
template <>
struct Vec<float, 4> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    float4 a = reinterpret_cast<const float4*>(p)[0];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
  static __device__ __forceinline__ void store(float* p, const float* v) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec<float, 2> {
  static __device__ __forceinline__ void load(const float* p, float* v) {
    float2 a = reinterpret_cast<const float2*>(p)[0];
    v[0] = a.x; v[1] = a.y;
  }
  static __device__ __forceinline__ void store(float* p, const float* v) {
    reinterpret_cast<float2*>(p)[0] = make_float2(v[0], v[1]);
  }
};
template <int ST>
struct Vec<double, ST> {
  static __device__ __forceinline__ void load(const double* p, double* v) {
#pragma unroll
    for (int i = 0; i < ST; i += 2) {
      double2 a = reinterpret_cast<const double2*>(p)[i / 2];
      v[i] = a.x;
      v[i + 1] = a.y;
    }
  }
  static __device__ __forceinline__ void store(double* p, const double* v) {
#pragma unroll
    for (int i = 0; i < ST; i += 2) reinterpret_cast<double2*>(p)[i / 2] = make_double2(v[i], v[i + 1]);
  }
};

template <int ST>
struct Vec<df64, ST> {
  static __device__ __forceinline__ void load(const df64* p, df64* v) {
#pragma unroll
    for (int i = 0; i < ST; i += 2) {
      const float4 a = reinterpret_cast<const float4*>(p)[i / 2];
      v[i] = df64(a.x, a.y);
      v[i + 1] = df64(a.z, a.w);
    }
  }
  static __device__ __forceinline__ void store(df64* p, const df64* v) {
#pragma unroll
    for (int i = 0; i < ST; i += 2)
      reinterpret_cast<float4*>(p)[i / 2] = make_float4(v[i].hi, v[i].lo, v[i + 1].hi, v[i + 1].lo);
  }
};

constexpr int kLG = 4;  // consecutive l per thread in the Legendre quadrature

// shared-memory footprint (elements of T) of one CTA
__host__ __device__ inline size_t rp_smem_elems(int L, int Q, int rowlen, int ST, int RC) {
  size_t L2 = (size_t)L * L, M2 = 2 * L - 1;
  return 2 * L2 * ST                    // Gs, Ga
         + (size_t)RC * 2 * M2 * ST     // Fb (F_j, F_jb, then A+, A-)
         + (size_t)RC * 4 * Q * ST      // Wb
         + (size_t)RC * rowlen          // Th
         + 2 * (size_t)L * Q;           // tc, ts
}

// One CTA's work: radial node k, states s0 .. s0+ST-1 of the block G ([k][lm][s], S columns).
template <typename T, int ST, int RC>
__device__ __forceinline__ void angular_rp_block(const AngArgs<T>& a, T* __restrict__ G, int k,
                                                 int s0, unsigned char* smem_raw) {
  const int L = a.L, lmax = L - 1, L2 = L * L, M2 = 2 * L - 1;
  const int Np = a.n_phi, h = Np / 2, Q4 = a.Q4, Q = Q4 + 1;
  const int Nt = a.n_theta, S = a.S, NP = (Nt + 1) / 2;
  const int rowlen = L * (L + 1) / 2;
  T* Gs = reinterpret_cast<T*>(smem_raw);
  T* Ga = Gs + (size_t)L2 * ST;
  T* Fb = Ga + (size_t)L2 * ST;
  T* Wb = Fb + (size_t)RC * 2 * M2 * ST;
  T* Th = Wb + (size_t)RC * 4 * Q * ST;
  T* tc = Th + (size_t)RC * rowlen;
  T* ts = tc + (size_t)L * Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = min(ST, S - s0);

  for (int i = tid; i < 2 * L * Q; i += RC * 32) tc[i] = a.trig[i];
  for (int i = tid; i < L2 * ST; i += RC * 32) {
    int lm = i / ST, s = i - lm * ST;
    Gs[i] = (s < ns) ? G[((size_t)k * L2 + lm) * S + s0 + s] : T(0);
    Ga[i] = T(0);
  }
  __syncthreads();

  T* F = Fb + (size_t)warp * 2 * M2 * ST;  // this warp's [2][M2][ST]
  T* Wf = Wb + (size_t)warp * 4 * Q * ST;  // this warp's [4][Q][ST]
  T* th = Th + (size_t)warp * rowlen;      // this warp's theta row
  const T* wvk = a.wv + (size_t)k * Nt * Np;

  for (int c0 = 0; c0 < NP; c0 += RC) {
    const int jp = c0 + warp;
    if (jp < NP) {
      const int jrow[2] = {jp, Nt - 1 - jp};
      const bool single = (jrow[0] == jrow[1]);
      for (int i = lane; i < rowlen; i += 32) th[i] = a.theta[(size_t)jp * rowlen + i];
      __syncwarp();
      // ---- Legendre sums (even / odd in l + |m|) for rows j and jb
      for (int mi = lane; mi < M2; mi += 32) {
        const int m = mi - lmax, am = m < 0 ? -m : m;
        const T* tr = th + theta_off(L, am) - am;
        T E[ST], O[ST], g[ST];
#pragma unroll
        for (int s = 0; s < ST; ++s) E[s] = O[s] = T(0);
        int l = am;
        for (; l + 1 <= lmax; l += 2) {
          T t0 = tr[l], t1 = tr[l + 1];
          Vec<T, ST>::load(Gs + (l * l + l + m) * ST, g);
#pragma unroll
          for (int s = 0; s < ST; ++s) E[s] = fma(t0, g[s], E[s]);
          Vec<T, ST>::load(Gs + ((l + 1) * (l + 1) + (l + 1) + m) * ST, g);
#pragma unroll
          for (int s = 0; s < ST; ++s) O[s] = fma(t1, g[s], O[s]);
        }
        if (l <= lmax) {
          T t0 = tr[l];
          Vec<T, ST>::load(Gs + (l * l + l + m) * ST, g);
#pragma unroll
          for (int s = 0; s < ST; ++s) E[s] = fma(t0, g[s], E[s]);
        }
#pragma unroll
        for (int s = 0; s < ST; ++s) {
          g[s] = E[s] + O[s];
          O[s] = E[s] - O[s];
        }
        Vec<T, ST>::store(F + (size_t)mi * ST, g);
        Vec<T, ST>::store(F + (size_t)(M2 + mi) * ST, O);
      }
      __syncwarp();
      const int nrows = single ? 1 : 2;
      for (int row = 0; row < nrows; ++row) {
        const T* Fr = F + (size_t)row * M2 * ST;
        const T* wvr = wvk + (size_t)jrow[row] * Np;
        // ---- phi sums at the folded angles, times W V, folded again for the quadrature
        for (int q = lane; q < Q; q += 32) {
          T Ee[ST], Eo[ST], Oe[ST], Oo[ST], fp[ST], fm[ST];
          Vec<T, ST>::load(Fr + (size_t)lmax * ST, Ee);
#pragma unroll
          for (int s = 0; s < ST; ++s) Eo[s] = Oe[s] = Oo[s] = T(0);
          int m = 1;
          for (; m + 1 <= lmax; m += 2) {
            T c1 = tc[m * Q + q], s1 = ts[m * Q + q];
            Vec<T, ST>::load(Fr + (size_t)(lmax + m) * ST, fp);
            Vec<T, ST>::load(Fr + (size_t)(lmax - m) * ST, fm);
#pragma unroll
            for (int s = 0; s < ST; ++s) {
              Eo[s] = fma(c1, fp[s], Eo[s]);
              Oo[s] = fma(s1, fm[s], Oo[s]);
            }
            T c2 = tc[(m + 1) * Q + q], s2 = ts[(m + 1) * Q + q];
            Vec<T, ST>::load(Fr + (size_t)(lmax + m + 1) * ST, fp);
            Vec<T, ST>::load(Fr + (size_t)(lmax - m - 1) * ST, fm);
#pragma unroll
            for (int s = 0; s < ST; ++s) {
              Ee[s] = fma(c2, fp[s], Ee[s]);
              Oe[s] = fma(s2, fm[s], Oe[s]);
            }
          }
          if (m <= lmax) {  // odd m left over
            T c1 = tc[m * Q + q], s1 = ts[m * Q + q];
            Vec<T, ST>::load(Fr + (size_t)(lmax + m) * ST, fp);
            Vec<T, ST>::load(Fr + (size_t)(lmax - m) * ST, fm);
#pragma unroll
            for (int s = 0; s < ST; ++s) {
              Eo[s] = fma(c1, fp[s], Eo[s]);
              Oo[s] = fma(s1, fm[s], Oo[s]);
            }
          }
          const int iq = q, iNq = (Np - q) % Np, ihm = h - q, ihp = h + q;
          const T w_q = wvr[iq], w_Nq = wvr[iNq], w_hm = wvr[ihm], w_hp = wvr[ihp];
          const T wq = (q == 0 || 2 * q == h) ? T(0.5) : T(1);
          T c0v[ST], c1v[ST], s0v[ST], s1v[ST];
#pragma unroll
          for (int s = 0; s < ST; ++s) {
            T EpE = Ee[s] + Eo[s], EmE = Ee[s] - Eo[s];
            T OpO = Oe[s] + Oo[s], OmO = Oe[s] - Oo[s];
            T g_q = w_q * (EpE + OpO);
            T g_Nq = w_Nq * (EpE - OpO);
            T g_hm = w_hm * (EmE - OmO);
            T g_hp = w_hp * (EmE + OmO);
            T P = wq * (g_q + g_Nq), Mm = wq * (g_q - g_Nq);
            T P2 = wq * (g_hm + g_hp), M2v = wq * (g_hm - g_hp);
            c0v[s] = P + P2;    // cos, even m
            c1v[s] = P - P2;    // cos, odd m
            s0v[s] = Mm - M2v;  // sin, even m
            s1v[s] = Mm + M2v;  // sin, odd m
          }
          Vec<T, ST>::store(Wf + (size_t)(0 * Q + q) * ST, c0v);
          Vec<T, ST>::store(Wf + (size_t)(1 * Q + q) * ST, c1v);
          Vec<T, ST>::store(Wf + (size_t)(2 * Q + q) * ST, s0v);
          Vec<T, ST>::store(Wf + (size_t)(3 * Q + q) * ST, s1v);
        }
        __syncwarp();
        // ---- phi quadrature: lane owns m; cos and sin coefficients
        for (int m = lane; m <= lmax; m += 32) {
          const T* srcc = Wf + (size_t)((m & 1) ? 1 : 0) * Q * ST;
          const T* srcs = Wf + (size_t)((m & 1) ? 3 : 2) * Q * ST;
          const T* tcm = tc + m * Q;
          const T* tsm = ts + m * Q;
          T Ac[ST], As[ST], v[ST];
#pragma unroll
          for (int s = 0; s < ST; ++s) Ac[s] = As[s] = T(0);
          for (int q = 0; q < Q; ++q) {
            T cq = tcm[q], sq = tsm[q];
            Vec<T, ST>::load(srcc + (size_t)q * ST, v);
#pragma unroll
            for (int s = 0; s < ST; ++s) Ac[s] = fma(cq, v[s], Ac[s]);
            Vec<T, ST>::load(srcs + (size_t)q * ST, v);
#pragma unroll
            for (int s = 0; s < ST; ++s) As[s] = fma(sq, v[s], As[s]);
          }
          // F rows are consumed: row 0 holds A_j, then A+ / A- after row 1
          T* a_c = F + (size_t)(lmax + m) * ST;
          T* a_s = F + (size_t)(lmax - m) * ST;
          if (row == 0) {
            Vec<T, ST>::store(a_c, Ac);
            if (m > 0) Vec<T, ST>::store(a_s, As);
            if (single) {
              Vec<T, ST>::store(a_c + (size_t)M2 * ST, Ac);
              if (m > 0) Vec<T, ST>::store(a_s + (size_t)M2 * ST, As);
            }
          } else {
            T aj[ST], p[ST];
            Vec<T, ST>::load(a_c, aj);
#pragma unroll
            for (int s = 0; s < ST; ++s) {
              p[s] = aj[s] + Ac[s];
              aj[s] = aj[s] - Ac[s];
            }
            Vec<T, ST>::store(a_c, p);
            Vec<T, ST>::store(a_c + (size_t)M2 * ST, aj);
            if (m > 0) {
              Vec<T, ST>::load(a_s, aj);
#pragma unroll
              for (int s = 0; s < ST; ++s) {
                p[s] = aj[s] + As[s];
                aj[s] = aj[s] - As[s];
              }
              Vec<T, ST>::store(a_s, p);
              Vec<T, ST>::store(a_s + (size_t)M2 * ST, aj);
            }
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // ---- Legendre quadrature over this chunk's row pairs: items (mi, l0 .. l0+kLG-1)
    const int nvalid = min(RC, NP - c0);
    const int ngroups_max = (L + kLG - 1) / kLG;
    for (int it = tid; it < M2 * ngroups_max; it += RC * 32) {
      const int mi = it / ngroups_max, grp = it - mi * ngroups_max;
      const int m = mi - lmax, am = m < 0 ? -m : m;
      const int l0 = am + grp * kLG;
      if (l0 > lmax) continue;
      const int cnt = min(kLG, lmax - l0 + 1);
      T acc[kLG][ST];
#pragma unroll
      for (int u = 0; u < kLG; ++u) {
        if (u < cnt) Vec<T, ST>::load(Ga + (size_t)((l0 + u) * (l0 + u) + (l0 + u) + m) * ST, acc[u]);
      }
      const int toff = theta_off(L, am) + (l0 - am);
      for (int w = 0; w < nvalid; ++w) {
        const T* Fw = Fb + (size_t)w * 2 * M2 * ST;
        T ap[ST], am_[ST];
        Vec<T, ST>::load(Fw + (size_t)mi * ST, ap);
        Vec<T, ST>::load(Fw + (size_t)(M2 + mi) * ST, am_);
        const T* thw = Th + (size_t)w * rowlen + toff;
#pragma unroll
        for (int u = 0; u < kLG; ++u) {
          if (u < cnt) {
            const T t = thw[u];
            const bool odd = ((l0 + u + am) & 1) != 0;
#pragma unroll
            for (int s = 0; s < ST; ++s) acc[u][s] = fma(t, odd ? am_[s] : ap[s], acc[u][s]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kLG; ++u) {
        if (u < cnt) Vec<T, ST>::store(Ga + (size_t)((l0 + u) * (l0 + u) + (l0 + u) + m) * ST, acc[u]);
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < L2 * ST; i += RC * 32) {
    int lm = i / ST, s = i - lm * ST;
    if (s < ns) G[((size_t)k * L2 + lm) * S + s0 + s] = Ga[i];
  }
}

}  // namespace cs
