// FP32 angular block of H.X (Sec. 2.2.2 eq. Ar_lm and the inverse transform of Sec. 2.2.4)
// organised as four register-blocked contractions per radial node (internal; used by
// angular_gm.cu and the batched kernel). Same arithmetic as the row-pair kernel: equatorial
// parity folding of the Legendre sums, four-angle folding of the phi sums, W V on the grid.
//
// A CTA owns radial node k and ST states and walks the theta rows in chunks of RC mirrored
// row pairs (Legendre rows staged transposed, [packed (m,l)][pair]). A column of the chunk is (pair p, row j or its mirror jb, state s):
// NC = 2 RC ST columns.
//   A: F[m][col]      = sum_l Theta_lm(t_j) G[l,m,s]            (even/odd l+|m| -> j, jb)
//   B: Wq[4][q][col]  = W V x the phi sums at the four mirror angles of q, folded back
//                       into cos/sin x even/odd-m quadrature inputs
//   C: A[m][col]      = sum_q {cos|sin}(m phi_q) Wq[...][q][col]
//   D: G'[l,m,s]     += sum_p Theta_lm(t_jp) (A_j +- A_jb)        (accumulated over chunks)
// Stages B and C (about 80 % of the flops) use 4 x 4 register tiles with the lanes of a
// warp laid out 4 (rows) x 8 (columns), so every 128-bit shared-memory load is shared by
// the lanes and feeds 8 (B) or 5 (C) FMAs per lane; stages A and D use 4 x 4 tiles over
// (l, pair or state).
#pragma once

#include <cuda_runtime.h>

#include "cs_internal.h"
#include "hx_kernels.cuh"

namespace cs {

constexpr int kGmThreads = 256;

__host__ __device__ inline int gm_round4(int x) { return (x + 3) & ~3; }

struct GmShape {
  int L, Q, Qp, Lp, rowlen, NC, NCp;
};

__host__ __device__ inline GmShape gm_shape(int L, int Q4, int ST, int RC) {
  GmShape g;
  g.L = L;
  g.Q = Q4 + 1;
  g.Qp = gm_round4(g.Q);
  g.Lp = gm_round4(L);
  g.rowlen = L * (L + 1) / 2;
  g.NC = 2 * RC * ST;
  g.NCp = g.NC % 32 == 0 ? g.NC + 4 : g.NC;  // F rows start on different banks
  return g;
}

// shared-memory footprint in bytes
__host__ __device__ inline size_t gm_smem_bytes(int L, int Q4, int ST, int RC) {
  const GmShape g = gm_shape(L, Q4, ST, RC);
  const size_t L2 = (size_t)L * L, M2 = 2 * L - 1;
  size_t f = 2 * L2 * ST + (size_t)RC * (g.rowlen + 4) + M2 * g.NCp +
             4 * (size_t)g.Qp * g.NC + 4 * (size_t)g.Lp * g.Qp;
  return f * sizeof(float);
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

template <int ST, int RC>
__device__ __forceinline__ void angular_gm_block(const AngArgs<float>& a, float* __restrict__ G,
                                                 int k, int s0, unsigned char* smem_raw) {
  static_assert(ST % 4 == 0 && RC % 4 == 0, "tiles of four");
  constexpr int NB = 8;  // global loads in flight per thread in the staging loops
  const int L = a.L, lmax = L - 1, L2 = L * L, M2 = 2 * L - 1;
  const int Np = a.n_phi, h = Np / 2, Q4 = a.Q4;
  const int Nt = a.n_theta, S = a.S, NP = (Nt + 1) / 2;
  const GmShape gs = gm_shape(L, Q4, ST, RC);
  const int Q = gs.Q, Qp = gs.Qp, Lp = gs.Lp, RL = gs.rowlen, NCp = gs.NCp;
  constexpr int NC = 2 * RC * ST;
  float* Gs = reinterpret_cast<float*>(smem_raw);      // [L2][ST]
  float* Ga = Gs + (size_t)L2 * ST;                    // [L2][ST]
  float* PT = Ga + (size_t)L2 * ST;                    // [RL + 4][RC]: packed (m,l) x pair
  float* F = PT + (size_t)(RL + 4) * RC;               // [M2][NCp] (A after stage C)
  float* Wq = F + (size_t)M2 * NCp;                    // [4][Qp][NC]
  float* Tb = Wq + (size_t)4 * Qp * NC;                // [cos|sin][Lp][Qp]
  float* Tc = Tb + (size_t)2 * Lp * Qp;                // [cos|sin][Qp][Lp]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = min(ST, S - s0);

  // ---- tables and the state tile of G (NB independent loads in flight per thread)
  for (int b0 = 0; b0 < 2 * Lp * Qp; b0 += NB * kGmThreads) {
    float v[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = b0 + u * kGmThreads + tid;
      v[u] = 0.f;
      if (i < 2 * Lp * Qp) {
        const int cs_ = i / (Lp * Qp), r = i - cs_ * Lp * Qp;
        const int m = r / Qp, q = r - m * Qp;
        if (m < L && q < Q) v[u] = a.trig[(size_t)(cs_ * L + m) * Q + q];
      }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = b0 + u * kGmThreads + tid;
      if (i < 2 * Lp * Qp) {
        const int cs_ = i / (Lp * Qp), r = i - cs_ * Lp * Qp;
        const int m = r / Qp, q = r - m * Qp;
        Tb[i] = v[u];
        Tc[(size_t)cs_ * Qp * Lp + q * Lp + m] = v[u];
      }
    }
  }
  for (int b0 = 0; b0 < L2 * ST; b0 += NB * kGmThreads) {
    float v[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = b0 + u * kGmThreads + tid;
      const int lm = i / ST, s = i - lm * ST;
      v[u] = (i < L2 * ST && s < ns) ? G[((size_t)k * L2 + lm) * S + s0 + s] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int i = b0 + u * kGmThreads + tid;
      if (i < L2 * ST) {
        Gs[i] = v[u];
        Ga[i] = 0.f;
      }
    }
  }
  for (int i = tid; i < 4 * RC; i += kGmThreads) PT[(size_t)RL * RC + i] = 0.f;
  const float* wvk = a.wv + (size_t)k * Nt * Np;

  for (int c0 = 0; c0 < NP; c0 += RC) {
    __syncthreads();  // set-up done / previous chunk's stage D done with PT and A
    // ---- theta rows of the chunk, transposed to [packed (m,l)][pair] (zero for missing pairs)
    for (int b0 = 0; b0 < RC * RL; b0 += NB * kGmThreads) {
      float v[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int i = b0 + u * kGmThreads + tid;
        const int p = i / RL, o = i - p * RL;
        v[u] = (i < RC * RL && c0 + p < NP) ? a.theta[(size_t)(c0 + p) * RL + o] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int i = b0 + u * kGmThreads + tid;
        const int p = i / RL, o = i - p * RL;
        if (i < RC * RL) PT[(size_t)o * RC + p] = v[u];
      }
    }
    __syncthreads();
    // ---- A: Legendre sums. Item = (mode, pair block, state block); modes in the order
    //      0, +1, -1, +2, -2, ... so that a warp's lanes have similar l ranges.
    {
      constexpr int NPB = RC / 4, NSB = ST / 4, NCMB = NPB * NSB;
      for (int it = tid; it < M2 * NCMB; it += kGmThreads) {
        const int mo = it / NCMB, cmb = it - mo * NCMB;
        const int pb = cmb / NSB, sb = cmb - pb * NSB;
        const int am = (mo + 1) >> 1, m = (mo & 1) ? am : -am;
        const int p0 = 4 * pb, s0l = 4 * sb;
        float E[4][4], O[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) E[u][v] = O[u][v] = 0.f;
        // rows (m, l) of PT for l = am, am+1, ... start at theta_off(L, am)
        const float* prow = PT + (size_t)theta_off(L, am) * RC + p0;
        for (int l0 = am; l0 <= lmax; l0 += 4) {
          float4 P4[4], g4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int l = l0 + i;
            P4[i] = ld4(prow + (size_t)(l - am) * RC);  // finite past lmax; multiplied by 0
            g4[i] = (l <= lmax) ? ld4(Gs + (size_t)(l * l + l + m) * ST + s0l)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float pv[4] = {P4[i].x, P4[i].y, P4[i].z, P4[i].w};
            const float gv[4] = {g4[i].x, g4[i].y, g4[i].z, g4[i].w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                if (i & 1) O[u][v] = fmaf(pv[u], gv[v], O[u][v]);
                else       E[u][v] = fmaf(pv[u], gv[v], E[u][v]);
              }
          }
        }
        const int mi = m + lmax;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float* fj = F + (size_t)mi * NCp + ((p0 + u) * 2) * ST + s0l;
          st4(fj, E[u][0] + O[u][0], E[u][1] + O[u][1], E[u][2] + O[u][2], E[u][3] + O[u][3]);
          st4(fj + ST, E[u][0] - O[u][0], E[u][1] - O[u][1], E[u][2] - O[u][2], E[u][3] - O[u][3]);
        }
      }
    }
    __syncthreads();
    // ---- B: phi sums at the folded angles, W V, folded quadrature inputs.
    //      Warp tile = 4 q-blocks x 8 column blocks (lanes 4 x 8).
    {
      const int nQB = Qp / 4, nQW = (nQB + 3) / 4;
      constexpr int nCW = NC / 32;
      for (int wt = warp; wt < nQW * nCW; wt += kGmThreads / 32) {
        const int qb = (wt % nQW) * 4 + (lane & 3);
        const int cb = (wt / nQW) * 8 + (lane >> 2);
        if (qb >= nQB) continue;
        const int q0 = 4 * qb, cc = 4 * cb;
        // the four columns share (pair, row): prefetch that row's W V at the 16 angles
        const int col_pr = cc / ST, p = col_pr >> 1, r = col_pr & 1;
        const int jp = c0 + p;
        const bool valid = (jp < NP) && !(r == 1 && (Nt - 1 - jp) == jp);
        const int jr = (r == 0) ? jp : Nt - 1 - jp;
        const float* wvr = wvk + (size_t)(valid ? jr : 0) * Np;
        float wang[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const bool ok = valid && q <= Q4;
          wang[i][0] = ok ? wvr[q] : 0.f;
          wang[i][1] = ok ? wvr[(Np - q) % Np] : 0.f;
          wang[i][2] = ok ? wvr[h - q] : 0.f;
          wang[i][3] = ok ? wvr[h + q] : 0.f;
        }
        float Ee[4][4], Eo[4][4], Oe[4][4], Oo[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) Ee[i][j] = Eo[i][j] = Oe[i][j] = Oo[i][j] = 0.f;
        for (int m = 0; m <= lmax; m += 2) {
          {
            const float4 tc4 = ld4(Tb + (size_t)m * Qp + q0);
            const float4 ts4 = ld4(Tb + (size_t)(Lp + m) * Qp + q0);
            const float4 fp4 = ld4(F + (size_t)(lmax + m) * NCp + cc);
            const float4 fm4 = ld4(F + (size_t)(lmax - m) * NCp + cc);
            const float tc[4] = {tc4.x, tc4.y, tc4.z, tc4.w}, ts[4] = {ts4.x, ts4.y, ts4.z, ts4.w};
            const float fp[4] = {fp4.x, fp4.y, fp4.z, fp4.w}, fm[4] = {fm4.x, fm4.y, fm4.z, fm4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                Ee[i][j] = fmaf(tc[i], fp[j], Ee[i][j]);
                Oe[i][j] = fmaf(ts[i], fm[j], Oe[i][j]);
              }
          }
          if (m + 1 <= lmax) {
            const int m1 = m + 1;
            const float4 tc4 = ld4(Tb + (size_t)m1 * Qp + q0);
            const float4 ts4 = ld4(Tb + (size_t)(Lp + m1) * Qp + q0);
            const float4 fp4 = ld4(F + (size_t)(lmax + m1) * NCp + cc);
            const float4 fm4 = ld4(F + (size_t)(lmax - m1) * NCp + cc);
            const float tc[4] = {tc4.x, tc4.y, tc4.z, tc4.w}, ts[4] = {ts4.x, ts4.y, ts4.z, ts4.w};
            const float fp[4] = {fp4.x, fp4.y, fp4.z, fp4.w}, fm[4] = {fm4.x, fm4.y, fm4.z, fm4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                Eo[i][j] = fmaf(tc[i], fp[j], Eo[i][j]);
                Oo[i][j] = fmaf(ts[i], fm[j], Oo[i][j]);
              }
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const float wq = (q == 0 || 2 * q == h) ? 0.5f : 1.f;
          float c0v[4], c1v[4], s0v[4], s1v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float EpE = Ee[i][j] + Eo[i][j], EmE = Ee[i][j] - Eo[i][j];
            const float OpO = Oe[i][j] + Oo[i][j], OmO = Oe[i][j] - Oo[i][j];
            const float g_q = wang[i][0] * (EpE + OpO), g_Nq = wang[i][1] * (EpE - OpO);
            const float g_hm = wang[i][2] * (EmE - OmO), g_hp = wang[i][3] * (EmE + OmO);
            const float Pp = wq * (g_q + g_Nq), Mm = wq * (g_q - g_Nq);
            const float P2 = wq * (g_hm + g_hp), M2v = wq * (g_hm - g_hp);
            c0v[j] = Pp + P2;
            c1v[j] = Pp - P2;
            s0v[j] = Mm - M2v;
            s1v[j] = Mm + M2v;
          }
          float* w0 = Wq + (size_t)q * NC + cc;
          st4(w0, c0v[0], c0v[1], c0v[2], c0v[3]);
          st4(w0 + (size_t)Qp * NC, c1v[0], c1v[1], c1v[2], c1v[3]);
          st4(w0 + (size_t)2 * Qp * NC, s0v[0], s0v[1], s0v[2], s0v[3]);
          st4(w0 + (size_t)3 * Qp * NC, s1v[0], s1v[1], s1v[2], s1v[3]);
        }
      }
    }
    __syncthreads();
    // ---- C: phi quadrature, A[+m] (cos) and A[-m] (sin), written over F.
    //      Warp tile = 4 m-blocks x 8 column blocks.
    {
      const int nMB = Lp / 4, nMW = (nMB + 3) / 4;
      constexpr int nCW = NC / 32;
      for (int wt = warp; wt < nMW * nCW; wt += kGmThreads / 32) {
        const int mb = (wt % nMW) * 4 + (lane & 3);
        const int cb = (wt / nMW) * 8 + (lane >> 2);
        if (mb >= nMB) continue;
        const int m0 = 4 * mb, cc = 4 * cb;
        float Ac[4][4], As[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) Ac[i][j] = As[i][j] = 0.f;
        for (int q = 0; q < Qp; ++q) {
          const float4 tc4 = ld4(Tc + (size_t)q * Lp + m0);
          const float4 ts4 = ld4(Tc + (size_t)(Qp + q) * Lp + m0);
          const float* wr = Wq + (size_t)q * NC + cc;
          const float4 we = ld4(wr), wo = ld4(wr + (size_t)Qp * NC);
          const float4 se = ld4(wr + (size_t)2 * Qp * NC), so = ld4(wr + (size_t)3 * Qp * NC);
          const float tc[4] = {tc4.x, tc4.y, tc4.z, tc4.w}, ts[4] = {ts4.x, ts4.y, ts4.z, ts4.w};
          const float ce[4] = {we.x, we.y, we.z, we.w}, co[4] = {wo.x, wo.y, wo.z, wo.w};
          const float sev[4] = {se.x, se.y, se.z, se.w}, sov[4] = {so.x, so.y, so.z, so.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              Ac[i][j] = fmaf(tc[i], (i & 1) ? co[j] : ce[j], Ac[i][j]);  // m0 is even
              As[i][j] = fmaf(ts[i], (i & 1) ? sov[j] : sev[j], As[i][j]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m = m0 + i;
          if (m > lmax) break;
          st4(F + (size_t)(lmax + m) * NCp + cc, Ac[i][0], Ac[i][1], Ac[i][2], Ac[i][3]);
          if (m > 0) st4(F + (size_t)(lmax - m) * NCp + cc, As[i][0], As[i][1], As[i][2], As[i][3]);
        }
      }
    }
    __syncthreads();
    // ---- D: Legendre quadrature. Item = (l block, mode, state block), l-block-major so
    //      that every item of a block has a non-empty l range; pairs taken four at a time.
    {
      constexpr int NSB = ST / 4;
      const int nLB = (L + 3) / 4;
      int total = 0;
      for (int lb = 0; lb < nLB && M2 - 8 * lb > 0; ++lb) total += (M2 - 8 * lb) * NSB;
      for (int it = tid; it < total; it += kGmThreads) {
        int rem = it, lb = 0;
        while (rem >= (M2 - 8 * lb) * NSB) {
          rem -= (M2 - 8 * lb) * NSB;
          ++lb;
        }
        const int mo = rem / NSB, sb = rem - mo * NSB;
        const int mi = 4 * lb + mo, m = mi - lmax, am = m < 0 ? -m : m;
        const int l0 = am + 4 * lb, s0l = 4 * sb;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int l = l0 + u;
          float4 v = (l <= lmax) ? ld4(Ga + (size_t)(l * l + l + m) * ST + s0l)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
          acc[u][0] = v.x; acc[u][1] = v.y; acc[u][2] = v.z; acc[u][3] = v.w;
        }
        const float* prow = PT + (size_t)(theta_off(L, am) + 4 * lb) * RC;
        const float* arow = F + (size_t)mi * NCp + s0l;
#pragma unroll
        for (int p4 = 0; p4 < RC; p4 += 4) {
          float pv[4][4];  // [u][pair]
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 t = ld4(prow + (size_t)u * RC + p4);
            pv[u][0] = t.x; pv[u][1] = t.y; pv[u][2] = t.z; pv[u][3] = t.w;
          }
#pragma unroll
          for (int pp = 0; pp < 4; ++pp) {
            const int p = p4 + pp;
            const float4 aj = ld4(arow + (size_t)(2 * p) * ST);
            const float4 ab = ld4(arow + (size_t)(2 * p + 1) * ST);
            const float ap[4] = {aj.x + ab.x, aj.y + ab.y, aj.z + ab.z, aj.w + ab.w};
            const float an[4] = {aj.x - ab.x, aj.y - ab.y, aj.z - ab.z, aj.w - ab.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v)
                acc[u][v] = fmaf(pv[u][pp], (u & 1) ? an[v] : ap[v], acc[u][v]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int l = l0 + u;
          if (l <= lmax)
            st4(Ga + (size_t)(l * l + l + m) * ST + s0l, acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < L2 * ST; i += kGmThreads) {
    const int lm = i / ST, s = i - lm * ST;
    if (s < ns) G[((size_t)k * L2 + lm) * S + s0 + s] = Ga[i];
  }
}

}  // namespace cs
