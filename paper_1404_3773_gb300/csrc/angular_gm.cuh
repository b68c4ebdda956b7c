// FP32 angular block of H.X (Sec. 2.2.2 eq. Ar_lm and the inverse transform of Sec. 2.2.4)
// organised as four register-blocked contractions per radial node (internal; used by
// angular_gm.cu and the batched kernel). Same arithmetic as the row-pair kernel: equatorial
// parity folding of the Legendre sums, four-angle folding of the phi sums, W V on the grid.
//
// A CTA owns radial node k and 8 states and walks the theta rows in chunks of 8 mirrored
// row pairs (p). Column of a chunk = (p, state pair sp, row r = j or its mirror jb, state
// e in the pair): col = 16 p + 4 sp + 2 r + e, so four consecutive columns hold both rows of
// two states and a thread can form A_j +- A_jb itself.
//   A: F[m][col]        = sum_l Theta_lm(t_j) G[l,m,s]           (even/odd l+|m| -> j, jb)
//   B: Wq[4][q][col]    = W V x the phi sums at the four mirror angles of q, folded back into
//                         cos/sin x even/odd-m quadrature inputs
//   C: AP[m][p][+-][s]  = sum_q {cos|sin}(m phi_q) Wq[...][q][col], combined over j, jb
//   D: G'[l,m][s]      += sum_p Theta_lm(t_jp) AP[m][p][parity of l+|m|][s]
// B and C use 4 x 4 register tiles with a warp's lanes laid out 4 (rows) x 8 (columns) and
// load the next step's operands while the current FMAs run; C groups the modes by parity
// so one tile needs one cos and one sin input array. D accumulates the (l, m) outputs for all
// 8 states in shared memory; an item is five l of one parity of one mode, its lanes share a
// mode, so each AP load is a broadcast that feeds 40 FMAs, and up to lmax 31 every thread has
// at most one item. The Legendre rows of a chunk come pre-transposed ([packed (m,l)][pair])
// from a table built at set-up, followed by the phi tables in their shared-memory layouts, so
// staging either is a contiguous copy. The W V rows of a chunk are staged in the AP region
// (free until stage C) before stage A. Both come from registers loaded during the previous
// chunk's stages C and D, so their global-memory latency overlaps that work; the state
// tile of G is fetched in a single round of loads.
#pragma once

#include <cuda_runtime.h>

#include "cs_internal.h"
#include "hx_kernels.cuh"

namespace cs {

constexpr int kGmThreads = 256;
constexpr int kGmST = 8;     // states per CTA
constexpr int kGmRC = 8;     // mirrored row pairs per chunk
constexpr int kGmItems = 2;  // Legendre-quadrature items per thread (up to 512 per CTA)
constexpr int kGmLq = 5;     // l per Legendre-quadrature item
constexpr int kGmPtRegs = 5;  // float4 of a chunk's Legendre rows per thread ((528+4) 8 / 4 / 256)
constexpr int kGmWvRegs = 8;  // W V values of a chunk per thread (16 (4 Q4 + 3) / 256, Q4 <= 31)
constexpr int kGmGRegs = 32;  // G-tile values per thread (32^2 8 / 256)

__host__ __device__ inline int gm_round4(int x) { return (x + 3) & ~3; }

struct GmShape {
  int L, Q, Qp, Lb, Lq, ne4, RL, NC, NCp, M2, nchunks;
};

__host__ __device__ inline GmShape gm_shape(int L, int Q4, int n_theta) {
  GmShape g;
  g.L = L;
  g.Q = Q4 + 1;
  g.Qp = gm_round4(g.Q);
  g.Lb = gm_round4(L + 1);
  g.ne4 = gm_round4((L + 1) / 2);         // even m = 0, 2, ... (padded), then odd m
  g.Lq = g.ne4 + gm_round4(L / 2);
  g.RL = L * (L + 1) / 2;
  g.NC = 2 * kGmRC * kGmST;
  g.NCp = g.NC + 4;                       // F rows start on different banks
  g.M2 = 2 * L - 1;
  g.nchunks = ((n_theta + 1) / 2 + kGmRC - 1) / kGmRC;
  return g;
}

// floats of the pre-transposed Legendre table: [chunk][RL + 4][kGmRC]
__host__ __device__ inline size_t gm_theta_pairs_elems(int L, int n_theta) {
  const GmShape g = gm_shape(L, 0, n_theta);
  return (size_t)g.nchunks * (g.RL + 4) * kGmRC;
}
// floats of the phi tables in their shared-memory layouts (Tb then Tc), stored after the
// Legendre table
__host__ __device__ inline size_t gm_trig_elems(int L, int Q4) {
  const GmShape g = gm_shape(L, Q4, 1);
  return 2 * (size_t)g.Lb * g.Qp + 2 * (size_t)(g.Qp + 1) * g.Lq;
}

// shared-memory footprint in bytes
__host__ __device__ inline size_t gm_smem_bytes(int L, int Q4, int n_theta) {
  const GmShape g = gm_shape(L, Q4, n_theta);
  const size_t L2 = (size_t)L * L;
  size_t f = 2 * L2 * kGmST + (size_t)(g.RL + 4) * kGmRC + (size_t)(g.M2 + 2) * g.NCp +
             (size_t)g.M2 * g.NC + 4 * (size_t)(g.Qp + 1) * g.NC + 2 * (size_t)g.Lb * g.Qp +
             2 * (size_t)(g.Qp + 1) * g.Lq;
  return f * sizeof(float) + (size_t)(g.M2 + 1) * sizeof(int);
}

// number of Legendre-quadrature items of angular_gm_block (four same-parity l of one mode)
__host__ __device__ inline int gm_items(int L) {
  int items = 0;
  for (int m = -(L - 1); m < L; ++m) {
    const int cnt = L - (m < 0 ? -m : m);
    items += ((cnt + 1) / 2 + kGmLq - 1) / kGmLq + (cnt / 2 + kGmLq - 1) / kGmLq;
  }
  return items;
}

// whether the block fits: shared memory, the per-thread item slots, and the W V rows of a
// chunk (2 kGmRC rows of n_phi <= 4 Q4 + 3 values) inside the AP region
__host__ __device__ inline bool gm_eligible(int L, int Q4, int n_theta) {
  const GmShape g = gm_shape(L, Q4, n_theta);
  return gm_smem_bytes(L, Q4, n_theta) <= 227 * 1024 && gm_items(L) <= kGmItems * kGmThreads &&
         (size_t)2 * kGmRC * (4 * Q4 + 4) <= (size_t)g.M2 * g.NC &&
         (g.RL + 4) * kGmRC / 4 <= kGmPtRegs * kGmThreads &&
         2 * kGmRC * (4 * Q4 + 3) <= kGmWvRegs * kGmThreads &&
         L * L * kGmST <= kGmGRegs * kGmThreads;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st2(float* p, float a, float b) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void unpack4(const float4 v, float* o) {
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}

__device__ __forceinline__ void angular_gm_block(const AngArgs<float>& a, float* __restrict__ G,
                                                 int k, int s0, unsigned char* smem_raw) {
  constexpr int ST = kGmST, RC = kGmRC, NC = 2 * RC * ST;
  const int L = a.L, lmax = L - 1, L2 = L * L, M2 = 2 * L - 1;
  const int Np = a.n_phi, h = Np / 2, Q4 = a.Q4;
  const int Nt = a.n_theta, S = a.S, NP = (Nt + 1) / 2;
  const GmShape gs = gm_shape(L, Q4, Nt);
  const int Q = gs.Q, Qp = gs.Qp, Lb = gs.Lb, Lq = gs.Lq, ne4 = gs.ne4, RL = gs.RL;
  const int NCp = gs.NCp;
  float* Gs = reinterpret_cast<float*>(smem_raw);  // [L2][ST]
  float* Ga = Gs + (size_t)L2 * ST;                // [L2][ST] Legendre-quadrature sums
  float* PT = Ga + (size_t)L2 * ST;                // [RL + 4][RC]
  float* Fz = PT + (size_t)(RL + 4) * RC;          // [M2 + 2][NCp], first and last rows zero
  float* F = Fz + NCp;                             // F[mi], mi in [-1, M2]
  float* AP = Fz + (size_t)(M2 + 2) * NCp;         // [M2][RC][2][ST]
  float* Wq = AP + (size_t)M2 * NC;                // [4][Qp + 1][NC], row Qp zero
  float* Tb = Wq + (size_t)4 * (Qp + 1) * NC;      // [cos|sin][Lb][Qp]
  float* Tc = Tb + (size_t)2 * Lb * Qp;            // [cos|sin][Qp + 1][Lq], m by parity
  int* mstart = reinterpret_cast<int*>(Tc + (size_t)2 * (Qp + 1) * Lq);  // [M2 + 1]
  const int WS = (Qp + 1) * NC;                    // stride of the four Wq arrays
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ns = min(ST, S - s0);

  // ---- set-up: phi tables (both layouts, from the set-up table), the state tile of G, zero
  //      rows, mode starts
  {
    const float4* src =
        reinterpret_cast<const float4*>(a.theta_pairs + gm_theta_pairs_elems(L, Nt));
    float4* dst = reinterpret_cast<float4*>(Tb);  // Tc follows Tb
    const int n4 = (int)(gm_trig_elems(L, Q4) / 4);
    for (int i = tid; i < n4; i += kGmThreads) dst[i] = src[i];
  }
  const float* wvk = a.wv + (size_t)k * Nt * Np;
  // the next chunk's Legendre rows and W V rows, held in registers until they are stored
  float4 pt_reg[kGmPtRegs];
  float wv_reg[kGmWvRegs];
  auto fetch_chunk = [&](int c, int chn) {
    const float4* src = reinterpret_cast<const float4*>(a.theta_pairs + (size_t)chn * (RL + 4) * RC);
    const int n4 = (RL + 4) * RC / 4;
#pragma unroll
    for (int u = 0; u < kGmPtRegs; ++u) {
      const int i = u * kGmThreads + tid;
      if (i < n4) pt_reg[u] = src[i];
    }
    const int n = RC * 2 * Np;
#pragma unroll
    for (int u = 0; u < kGmWvRegs; ++u) {
      const int i = u * kGmThreads + tid;
      float v = 0.f;
      if (i < n) {
        const int pr = i / Np, q = i - pr * Np;
        const int p = pr >> 1, r = pr & 1;
        const int jp = c + p;
        const int row = r ? Nt - 1 - jp : jp;
        if (jp < NP && (r == 0 || row != jp)) v = wvk[(size_t)row * Np + q];
      }
      wv_reg[u] = v;
    }
  };
  // the state tile of G in one round of loads, together with the first chunk's rows
  {
    float v[kGmGRegs];
#pragma unroll
    for (int u = 0; u < kGmGRegs; ++u) {
      const int i = u * kGmThreads + tid;
      const int lm = i / ST, s = i - lm * ST;
      v[u] = (i < L2 * ST && s < ns) ? G[((size_t)k * L2 + lm) * S + s0 + s] : 0.f;
    }
    fetch_chunk(0, 0);
#pragma unroll
    for (int u = 0; u < kGmGRegs; ++u) {
      const int i = u * kGmThreads + tid;
      if (i < L2 * ST) {
        Gs[i] = v[u];
        Ga[i] = 0.f;
      }
    }
  }
  for (int i = tid; i < NCp; i += kGmThreads) {
    Fz[i] = 0.f;
    Fz[(size_t)(M2 + 1) * NCp + i] = 0.f;
  }
  for (int i = tid; i < 4 * NC; i += kGmThreads) Wq[(size_t)(i / NC) * WS + (size_t)Qp * NC + i % NC] = 0.f;
  // Legendre-quadrature items: (mode, parity of l - |m|, group of kGmLq such l); mstart[mi] is the
  // first item of mode mi, the even-parity groups first
  if (tid == 0) {
    int o = 0;
    for (int mi = 0; mi < M2; ++mi) {
      mstart[mi] = o;
      const int m = mi - lmax, cnt = L - (m < 0 ? -m : m);
      o += ((cnt + 1) / 2 + kGmLq - 1) / kGmLq + (cnt / 2 + kGmLq - 1) / kGmLq;
    }
    mstart[M2] = o;
  }
  __syncthreads();
  const int nitems = mstart[M2];
  int item_code[kGmItems];  // mi | parity << 8 | group << 9, or -1
#pragma unroll
  for (int u = 0; u < kGmItems; ++u) {
    const int t = tid + u * kGmThreads;
    item_code[u] = -1;
    if (t < nitems) {
      int lo = 0, hi = M2 - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mstart[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      const int m = lo - lmax, cnt = L - (m < 0 ? -m : m);
      const int ge = ((cnt + 1) / 2 + kGmLq - 1) / kGmLq;  // even-parity groups of this mode
      const int r = t - mstart[lo];
      item_code[u] = (r < ge) ? (lo | (r << 9)) : (lo | (1 << 8) | ((r - ge) << 9));
    }
  }

  for (int c0 = 0, ch = 0; c0 < NP; c0 += RC, ++ch) {
    __syncthreads();  // previous chunk's stage D done with PT and AP
    // ---- the chunk's Legendre rows (pre-transposed table) and its pairs' W V rows into the
    //      AP region (unused until stage C): WVs[p][r][q], r = 0 row j = c0 + p, r = 1 its
    //      mirror; zero where absent. Both were fetched into registers earlier.
    {
      float4* dst = reinterpret_cast<float4*>(PT);
      const int n4 = (RL + 4) * RC / 4;
#pragma unroll
      for (int u = 0; u < kGmPtRegs; ++u) {
        const int i = u * kGmThreads + tid;
        if (i < n4) dst[i] = pt_reg[u];
      }
      const int n = RC * 2 * Np;
#pragma unroll
      for (int u = 0; u < kGmWvRegs; ++u) {
        const int i = u * kGmThreads + tid;
        if (i < n) AP[i] = wv_reg[u];
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
        const float* prow = PT + (size_t)theta_off(L, am) * RC + p0;
        for (int l0 = am; l0 <= lmax; l0 += 4) {
          float4 P4[4], g4[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int l = l0 + i;
            P4[i] = ld4(prow + (size_t)(l - am) * RC);  // finite past lmax; times 0 below
            g4[i] = (l <= lmax) ? ld4(Gs + (size_t)(l * l + l + m) * ST + s0l)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float pv[4], gv[4];
            unpack4(P4[i], pv);
            unpack4(g4[i], gv);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                if (i & 1) O[u][v] = fmaf(pv[u], gv[v], O[u][v]);
                else       E[u][v] = fmaf(pv[u], gv[v], E[u][v]);
              }
          }
        }
        float* frow = F + (size_t)(m + lmax) * NCp + 2 * s0l;  // state pair sp = s0l / 2
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float* f = frow + (size_t)(p0 + u) * 16;
          st4(f, E[u][0] + O[u][0], E[u][1] + O[u][1], E[u][0] - O[u][0], E[u][1] - O[u][1]);
          st4(f + 4, E[u][2] + O[u][2], E[u][3] + O[u][3], E[u][2] - O[u][2], E[u][3] - O[u][3]);
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
        float Ee[4][4], Eo[4][4], Oe[4][4], Oo[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) Ee[i][j] = Eo[i][j] = Oe[i][j] = Oo[i][j] = 0.f;
        // operands of mode m are loaded while the other parity's FMAs run; rows past lmax
        // are zero padding, so the odd partner of the last even mode needs no test
        float4 e_tc = ld4(Tb + q0), e_ts = ld4(Tb + (size_t)Lb * Qp + q0);
        float4 e_fp = ld4(F + (size_t)lmax * NCp + cc), e_fm = e_fp;
        for (int m = 0; m < L; m += 2) {
          const int mo = m + 1;
          const float4 o_tc = ld4(Tb + (size_t)mo * Qp + q0);
          const float4 o_ts = ld4(Tb + (size_t)(Lb + mo) * Qp + q0);
          const float4 o_fp = ld4(F + (size_t)(lmax + mo) * NCp + cc);
          const float4 o_fm = ld4(F + (size_t)(lmax - mo) * NCp + cc);
          {
            float tc[4], ts[4], fp[4], fm[4];
            unpack4(e_tc, tc); unpack4(e_ts, ts); unpack4(e_fp, fp); unpack4(e_fm, fm);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                Ee[i][j] = fmaf(tc[i], fp[j], Ee[i][j]);
                Oe[i][j] = fmaf(ts[i], fm[j], Oe[i][j]);
              }
          }
          if (m + 2 < L) {
            const int me = m + 2;
            e_tc = ld4(Tb + (size_t)me * Qp + q0);
            e_ts = ld4(Tb + (size_t)(Lb + me) * Qp + q0);
            e_fp = ld4(F + (size_t)(lmax + me) * NCp + cc);
            e_fm = ld4(F + (size_t)(lmax - me) * NCp + cc);
          }
          {
            float tc[4], ts[4], fp[4], fm[4];
            unpack4(o_tc, tc); unpack4(o_ts, ts); unpack4(o_fp, fp); unpack4(o_fm, fm);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                Eo[i][j] = fmaf(tc[i], fp[j], Eo[i][j]);
                Oo[i][j] = fmaf(ts[i], fm[j], Oo[i][j]);
              }
          }
        }
        // W V of the pair's two rows at the 16 angles of the tile (staged rows; zero rows
        // stand for absent mirrors and pairs past the last)
        const int p = cb >> 2;  // 4 column blocks per pair
        const float* wr0 = AP + (size_t)(2 * p) * Np;
        const float* wr1 = wr0 + Np;
        float wang[2][4][4];  // [row][q][angle q, N-q, h-q, h+q]
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const bool ok = q <= Q4;
          const int i0 = q, i1 = (Np - q) % Np, i2 = h - q, i3 = h + q;
          wang[0][i][0] = ok ? wr0[i0] : 0.f;
          wang[0][i][1] = ok ? wr0[i1] : 0.f;
          wang[0][i][2] = ok ? wr0[i2] : 0.f;
          wang[0][i][3] = ok ? wr0[i3] : 0.f;
          wang[1][i][0] = ok ? wr1[i0] : 0.f;
          wang[1][i][1] = ok ? wr1[i1] : 0.f;
          wang[1][i][2] = ok ? wr1[i2] : 0.f;
          wang[1][i][3] = ok ? wr1[i3] : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int q = q0 + i;
          const float wq = (q == 0 || 2 * q == h) ? 0.5f : 1.f;
          float c0v[4], c1v[4], s0v[4], s1v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = j >> 1;  // columns 0,1: row j; 2,3: mirror row jb
            const float EpE = Ee[i][j] + Eo[i][j], EmE = Ee[i][j] - Eo[i][j];
            const float OpO = Oe[i][j] + Oo[i][j], OmO = Oe[i][j] - Oo[i][j];
            const float g_q = wang[r][i][0] * (EpE + OpO), g_Nq = wang[r][i][1] * (EpE - OpO);
            const float g_hm = wang[r][i][2] * (EmE - OmO), g_hp = wang[r][i][3] * (EmE + OmO);
            const float Pp = wq * (g_q + g_Nq), Mm = wq * (g_q - g_Nq);
            const float P2 = wq * (g_hm + g_hp), M2v = wq * (g_hm - g_hp);
            c0v[j] = Pp + P2;
            c1v[j] = Pp - P2;
            s0v[j] = Mm - M2v;
            s1v[j] = Mm + M2v;
          }
          float* w0 = Wq + (size_t)q * NC + cc;
          st4(w0, c0v[0], c0v[1], c0v[2], c0v[3]);
          st4(w0 + WS, c1v[0], c1v[1], c1v[2], c1v[3]);
          st4(w0 + 2 * (size_t)WS, s0v[0], s0v[1], s0v[2], s0v[3]);
          st4(w0 + 3 * (size_t)WS, s1v[0], s1v[1], s1v[2], s1v[3]);
        }
      }
    }
    __syncthreads();
    // the next chunk's rows: their loads run while stages C and D compute
    if (c0 + RC < NP) fetch_chunk(c0 + RC, ch + 1);
    // ---- C: phi quadrature of one parity class of modes per tile, combined over the mirror
    //      rows: AP[m][p][0] = A_j + A_jb, AP[m][p][1] = A_j - A_jb. Warp tile = 4 mode
    //      blocks x 8 column blocks.
    {
      const int nMB = Lq / 4, nMW = (nMB + 3) / 4;
      constexpr int nCW = NC / 32;
      for (int wt = warp; wt < nMW * nCW; wt += kGmThreads / 32) {
        const int mb = (wt % nMW) * 4 + (lane & 3);
        const int cb = (wt / nMW) * 8 + (lane >> 2);
        if (mb >= nMB) continue;
        const int mp0 = 4 * mb, cc = 4 * cb;
        const int par = (mp0 >= ne4) ? 1 : 0;
        const float* wc = Wq + (size_t)par * WS + cc;         // cos, parity of m
        const float* wsn = Wq + (size_t)(2 + par) * WS + cc;  // sin, parity of m
        float Ac[4][4], As[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) Ac[i][j] = As[i][j] = 0.f;
        // row Qp of Tc and Wq is zero, so the prefetch of step q + 1 needs no test
        float4 c_tc = ld4(Tc + mp0), c_ts = ld4(Tc + (size_t)(Qp + 1) * Lq + mp0);
        float4 c_wc = ld4(wc), c_ws = ld4(wsn);
        for (int q = 0; q < Qp; ++q) {
          const float4 n_tc = ld4(Tc + (size_t)(q + 1) * Lq + mp0);
          const float4 n_ts = ld4(Tc + (size_t)(Qp + 1 + q + 1) * Lq + mp0);
          const float4 n_wc = ld4(wc + (size_t)(q + 1) * NC);
          const float4 n_ws = ld4(wsn + (size_t)(q + 1) * NC);
          float tc[4], ts[4], w1[4], w2[4];
          unpack4(c_tc, tc); unpack4(c_ts, ts); unpack4(c_wc, w1); unpack4(c_ws, w2);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              Ac[i][j] = fmaf(tc[i], w1[j], Ac[i][j]);
              As[i][j] = fmaf(ts[i], w2[j], As[i][j]);
            }
          c_tc = n_tc; c_ts = n_ts; c_wc = n_wc; c_ws = n_ws;
        }
        const int p = cb >> 2, sp = cb & 3;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int mp = mp0 + i;
          const int m = par ? 2 * (mp - ne4) + 1 : 2 * mp;
          if (m > lmax) continue;
          float* ac = AP + ((size_t)(lmax + m) * RC + p) * 2 * ST + 2 * sp;
          st2(ac, Ac[i][0] + Ac[i][2], Ac[i][1] + Ac[i][3]);
          st2(ac + ST, Ac[i][0] - Ac[i][2], Ac[i][1] - Ac[i][3]);
          if (m > 0) {
            float* as = AP + ((size_t)(lmax - m) * RC + p) * 2 * ST + 2 * sp;
            st2(as, As[i][0] + As[i][2], As[i][1] + As[i][3]);
            st2(as + ST, As[i][0] - As[i][2], As[i][1] - As[i][3]);
          }
        }
      }
    }
    __syncthreads();
    // ---- D: Legendre quadrature. Item = kGmLq l of one parity (l - |m| = par, par + 2, ...)
    //      of one mode: they read the same half of AP, so each broadcast AP load feeds
    //      8 kGmLq FMAs.
#pragma unroll
    for (int u = 0; u < kGmItems; ++u) {
      const int code = item_code[u];
      if (code < 0) continue;
      const int mi = code & 0xff, par = (code >> 8) & 1, grp = code >> 9;
      const int m = mi - lmax, am = m < 0 ? -m : m;
      const int lbase = am + par + 2 * kGmLq * grp;  // l_v = lbase + 2 v
      float acc[kGmLq][ST], pv[kGmLq][RC];
#pragma unroll
      for (int v = 0; v < kGmLq; ++v) {
        const int l = lbase + 2 * v;
        if (l <= lmax) {
          const float* ga = Ga + (size_t)(l * l + l + m) * ST;
          unpack4(ld4(ga), acc[v]);
          unpack4(ld4(ga + 4), acc[v] + 4);
          const float* pr = PT + (size_t)(theta_off(L, am) + l - am) * RC;
          unpack4(ld4(pr), pv[v]);
          unpack4(ld4(pr + 4), pv[v] + 4);
        } else {
#pragma unroll
          for (int q = 0; q < ST; ++q) acc[v][q] = 0.f;
#pragma unroll
          for (int q = 0; q < RC; ++q) pv[v][q] = 0.f;
        }
      }
      const float* arow = AP + (size_t)mi * RC * 2 * ST + (par ? ST : 0);
#pragma unroll
      for (int pp = 0; pp < RC; ++pp) {
        float av[ST];
        unpack4(ld4(arow + (size_t)pp * 2 * ST), av);
        unpack4(ld4(arow + (size_t)pp * 2 * ST + 4), av + 4);
#pragma unroll
        for (int v = 0; v < kGmLq; ++v)
#pragma unroll
          for (int q = 0; q < ST; ++q) acc[v][q] = fmaf(pv[v][pp], av[q], acc[v][q]);
      }
#pragma unroll
      for (int v = 0; v < kGmLq; ++v) {
        const int l = lbase + 2 * v;
        if (l > lmax) break;
        float* ga = Ga + (size_t)(l * l + l + m) * ST;
        st4(ga, acc[v][0], acc[v][1], acc[v][2], acc[v][3]);
        st4(ga + 4, acc[v][4], acc[v][5], acc[v][6], acc[v][7]);
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < L2 * ST; i += kGmThreads) {
    const int lm = i / ST, sl = i - lm * ST;
    if (sl < ns) G[((size_t)k * L2 + lm) * S + s0 + sl] = Ga[i];
  }
}

}  // namespace cs
