// Angular block of H.X (Sec. 2.2.2 eq. Ar_lm and the inverse transform of Sec. 2.2.4) for the
// mixed-precision filter: the two phi transforms run on the 5th-generation tensor cores
// (tcgen05), the two Legendre contractions on the FP32 pipe.
//
// A CTA owns radial node k and 8 states and walks the theta rows in chunks of 8 mirrored row
// pairs, as the register-blocked FP32 kernel (angular_gm.cuh) does, with the same 128 columns
// col = 16 p + 4 sp + 2 r + e (pair p, state pair sp, row r = j or its mirror jb, state e of
// the pair). Per chunk:
//   A   (FP32)  F[col][kap]  = sum_l Theta_lm(t_row) G[l,m,s], kap = m + lmax, stored as FP32
//               rows, then converted to split BF16 (hi = bf16(x), lo = bf16(x - hi)) in the
//               MMA's A operand by a pass whose 16-byte stores are free of bank conflicts
//   B   (MMA)   D_B[col][p]  = sum_kap F[col][kap] T[p][kap], T[p][kap] = cos(m phi_p) for
//               m >= 0 and sin(|m| phi_p) for m < 0: the grid values on all n_phi angles
//   epi         g[col][p]    = W V(k, row, p) D_B[col][p], split BF16, into the next A operand
//   C   (MMA)   D_C[col][kap] = sum_p g[col][p] T[p][kap]: the phi quadrature
//   epi         AP[kap][p][+-][s] = D_C of row j +- D_C of row jb (a lane shuffle)
//   D   (FP32)  G'[l,m][s]  += sum_pairs Theta_lm(t_j) AP[...]: a thread owns one item of 5
//               same-parity l of one mode, keeps its sums in registers for the whole tile and
//               writes them to G at the tile's end
// The phi sums are plain dense products over all n_phi angles (no folding of the four mirror
// angles), which costs the tensor cores nothing and keeps the epilogues elementwise.
// The MMA operands are BF16 in the canonical K-major no-swizzle layout; each product is
// accumulated in FP32 tensor memory as hi*hi + hi*lo + lo*hi (split BF16, about 16
// significant bits). The FP32 F rows with the F operand, the g operand, and AP share one
// shared-memory region: each is dead once the pass or the MMA that reads it has completed.
// The two trig operands (T as B of the first MMA; T transposed, hi rows stacked over lo rows,
// as B of the second) are pre-split and pre-laid-out at set-up and copied once per CTA by the
// TMA engine (cp.async.bulk). CTAs are persistent (one per SM) and loop over the tiles.
// Every mbarrier wait is bounded: on expiry the kernel records an error code in a device word,
// releases its tensor memory and returns without writing G.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "angular_gm.cuh"
#include "cs_internal.h"
#include "hx_kernels.cuh"
#include "tc_common.cuh"

namespace cs {

namespace {

using namespace tcx;

constexpr int kTaThreads = 256;
constexpr int kST = kGmST;            // states per CTA
constexpr int kRC = kGmRC;            // mirrored row pairs per chunk
constexpr int kNC = 2 * kRC * kST;    // columns per chunk = MMA M
static_assert(kNC == 128, "the chunk's columns are the MMA's 128 rows");
constexpr int kNCp = kNC + 4;         // FP32 F row stride (rows start on different banks)
constexpr int kAPS = kNC + 4;         // AP stride per mode (stage D's lanes on different modes
                                      // then read different banks)
// The next chunk's Legendre rows and W V rows are fetched into registers by warps 1..7 only, so
// that warp 0 issues the MMAs without waiting on that work.
constexpr int kFetchThreads = kTaThreads - 32;
constexpr int kTaPtRegs = 5;   // float4 of Legendre rows per fetching thread ((528+4) 8 / 4 / 224)
constexpr int kTaWvRegs = 10;  // W V values per fetching thread (2 8 n_phi / 224, n_phi <= 140)

__host__ __device__ inline int round32(int x) { return (x + 31) & ~31; }
__host__ __device__ inline int round64(int x) { return (x + 63) & ~63; }

// split BF16 of two values, packed: hi = bf16x2(a, b), lo = bf16x2(a - hi.a, b - hi.b)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

struct TaShape {
  int M2, Kb, NB, RL, NP;
  // byte offsets in dynamic shared memory
  size_t off_tb, off_tc, off_x, off_gs, off_pt, off_wv, off_ms, total;
};

// Kb = modes rounded up to 32 (split into 16-column tensor-memory loads between the two warps
// of a lane quarter), NB = angles rounded up to 64 (32-column loads)
__host__ __device__ inline TaShape ta_shape(int L, int n_theta, int n_phi) {
  TaShape s;
  s.M2 = 2 * L - 1;
  s.Kb = round32(s.M2);
  s.NB = round64(n_phi);
  s.RL = L * (L + 1) / 2;
  s.NP = (n_theta + 1) / 2;
  size_t o = 0;
  s.off_tb = o;
  o += (size_t)2 * s.NB * s.Kb * 2;  // T (rows p, K = kap), hi then lo
  s.off_tc = o;
  o += (size_t)2 * s.Kb * s.NB * 2;  // T^T: rows kap (hi) then Kb + kap (lo), K = p
  s.off_x = o;
  // F operand followed by the FP32 F rows it is converted from ([M2][kNCp])
  size_t xb = (size_t)2 * kNC * s.Kb * 2 + (size_t)s.M2 * kNCp * 4;
  if ((size_t)2 * kNC * s.NB * 2 > xb) xb = (size_t)2 * kNC * s.NB * 2;  // g operand
  if ((size_t)s.M2 * kAPS * 4 > xb) xb = (size_t)s.M2 * kAPS * 4;          // AP
  o += xb;
  s.off_gs = o;
  o += (size_t)L * L * kST * 4;
  s.off_pt = o;
  o += (size_t)(s.RL + 4) * kRC * 4;
  s.off_wv = o;
  o += (size_t)2 * kRC * n_phi * 4;
  o = (o + 15) & ~(size_t)15;
  s.off_ms = o;
  o += (size_t)(s.M2 + 1) * 4;
  s.total = o;
  return s;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// src_bytes = 0 fills the destination word with zero and reads nothing
__device__ __forceinline__ void cp_async4(uint32_t dst, const float* src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__host__ __device__ inline uint32_t ta_tmem_cols(int NB, int Kb) {
  uint32_t c = 32;
  while ((int)c < NB + Kb) c <<= 1;
  return c;
}

__global__ void __launch_bounds__(kTaThreads, 1)
    k_angular_tc(AngArgs<float> a, const __nv_bfloat16* __restrict__ tphi,
                 float* __restrict__ G, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base_sh;
  constexpr int ST = kST, RC = kRC, NC = kNC;
  const int L = a.L, lmax = L - 1, L2 = L * L, M2 = 2 * L - 1;
  const int Np = a.n_phi, Nt = a.n_theta, S = a.S;
  const TaShape sh = ta_shape(L, Nt, Np);
  const int Kb = sh.Kb, NB = sh.NB, RL = sh.RL, NP = sh.NP;
  unsigned char* Fhi = smem + sh.off_x;                 // F operand: NC x Kb, hi then lo
  unsigned char* Flo = Fhi + (size_t)NC * Kb * 2;
  unsigned char* Ghi = smem + sh.off_x;                 // g operand: NC x NB, hi then lo
  unsigned char* Glo = Ghi + (size_t)NC * NB * 2;
  float* F32 = reinterpret_cast<float*>(Flo + (size_t)NC * Kb * 2);  // [M2][kNCp]
  float* AP = reinterpret_cast<float*>(smem + sh.off_x);  // [M2][kAPS]: [RC][2][ST] + pad
  float* Gs = reinterpret_cast<float*>(smem + sh.off_gs);  // [L2][ST]
  float* PT = reinterpret_cast<float*>(smem + sh.off_pt);  // [RL + 4][RC]
  float* WV = reinterpret_cast<float*>(smem + sh.off_wv);  // [RC][2][Np]
  int* mstart = reinterpret_cast<int*>(smem + sh.off_ms);  // [M2 + 1]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // tiles t = (radial node t / nst, states (t % nst) ST ..), taken in steps of the grid size
  const int nst = (S + ST - 1) / ST, ntiles = nst * a.n_r;
  const uint32_t bar_tma = smem_u32(&bars[0]);
  const uint32_t bar_mma = smem_u32(&bars[1]);
  const uint32_t tcols = ta_tmem_cols(NB, 2 * Kb);
  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base_sh), tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  // both trig operands in one bulk copy (their set-up image is the start of shared memory)
  if (tid == 0) {
    mbar_expect_tx(bar_tma, (uint32_t)sh.off_x);
    bulk_g2s(smem_u32(smem + sh.off_tb), tphi, (uint32_t)sh.off_x, bar_tma);
  }

  const int ft = tid - 32;  // fetching thread, warps 1..7
  float4 pt_reg[kTaPtRegs];
  float wv_reg[kTaWvRegs];
  // W V element u of this thread: staged index ft + u kFetchThreads = pr Np + q, packed as
  // pr << 16 | q once per CTA (-1 past the end)
  int wv_pq[kTaWvRegs];
#pragma unroll
  for (int u = 0; u < kTaWvRegs; ++u) {
    const int i = u * kFetchThreads + ft;
    wv_pq[u] = -1;
    if (ft >= 0 && i < RC * 2 * Np) {
      const int pr = i / Np;
      wv_pq[u] = (pr << 16) | (i - pr * Np);
    }
  }
  auto fetch_chunk = [&](const float* wvk, int c, int chn) {
    if (ft < 0) return;
    const float4* src =
        reinterpret_cast<const float4*>(a.theta_pairs + (size_t)chn * (RL + 4) * RC);
    const int n4 = (RL + 4) * RC / 4;
#pragma unroll
    for (int u = 0; u < kTaPtRegs; ++u) {
      const int i = u * kFetchThreads + ft;
      if (i < n4) pt_reg[u] = src[i];
    }
#pragma unroll
    for (int u = 0; u < kTaWvRegs; ++u) {
      float v = 0.f;
      if (wv_pq[u] >= 0) {
        const int pr = wv_pq[u] >> 16, q = wv_pq[u] & 0xffff;
        const int jp = c + (pr >> 1);
        const int row = (pr & 1) ? Nt - 1 - jp : jp;
        if (jp < NP && ((pr & 1) == 0 || row != jp)) v = wvk[(size_t)row * Np + q];
      }
      wv_reg[u] = v;
    }
  };
  // the next tile's state tile of G, streamed into Gs by cp.async (zero fill past the states)
  auto prefetch_g = [&](int kn, int s0n) {
    const int nsn = min(ST, S - s0n);
    if ((S & 3) == 0 && nsn == ST && (reinterpret_cast<uintptr_t>(G) & 15) == 0) {
      for (int i = tid; i < L2 * 2; i += kTaThreads) {
        const int lm = i >> 1, h = i & 1;
        cp_async16(smem_u32(Gs + lm * ST + 4 * h), G + ((size_t)kn * L2 + lm) * S + s0n + 4 * h);
      }
    } else {
      for (int i = tid; i < L2 * ST; i += kTaThreads) {
        const int lm = i / ST, sl = i - lm * ST;
        const bool in = sl < nsn;
        cp_async4(smem_u32(Gs + i), in ? G + ((size_t)kn * L2 + lm) * S + s0n + sl : G, in ? 4 : 0);
      }
    }
    cp_async_commit();
  };
  {
    const int k = blockIdx.x / nst, s0 = (blockIdx.x % nst) * ST, ns = min(ST, S - s0);
    float v[kGmGRegs];
#pragma unroll
    for (int u = 0; u < kGmGRegs; ++u) {
      const int i = u * kTaThreads + tid;
      const int lm = i / ST, s = i - lm * ST;
      v[u] = (i < L2 * ST && s < ns) ? G[((size_t)k * L2 + lm) * S + s0 + s] : 0.f;
    }
    fetch_chunk(a.wv + (size_t)k * Nt * Np, 0, 0);
#pragma unroll
    for (int u = 0; u < kGmGRegs; ++u) {
      const int i = u * kTaThreads + tid;
      if (i < L2 * ST) Gs[i] = v[u];
    }
  }
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
  // this thread's Legendre-quadrature item (at most one per thread): mode mi, parity of
  // l - |m|, group of kGmLq such l; its sums stay in registers for the whole tile
  int d_mi = 0, d_m = 0, d_am = 0, d_lbase = 0, d_par = 0;
  bool d_live = false;
  if (tid < nitems) {
    int lo = 0, hi = M2 - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (mstart[mid] <= tid) lo = mid;
      else hi = mid - 1;
    }
    const int m = lo - lmax, cnt = L - (m < 0 ? -m : m);
    const int ge = ((cnt + 1) / 2 + kGmLq - 1) / kGmLq;
    const int r = tid - mstart[lo];
    d_mi = lo;
    d_m = m;
    d_am = m < 0 ? -m : m;
    d_par = (r < ge) ? 0 : 1;
    d_lbase = d_am + d_par + 2 * kGmLq * ((r < ge) ? r : r - ge);  // l_v = d_lbase + 2 v
    d_live = true;
  }
  float dacc[kGmLq][ST];
#pragma unroll
  for (int v = 0; v < kGmLq; ++v)
#pragma unroll
    for (int q = 0; q < ST; ++q) dacc[v][q] = 0.f;
  bool ok = mbar_wait(bar_tma, 0);
  if (!ok) atomicCAS(err, 0, 1);
  ok = __syncthreads_and(ok ? 1 : 0) != 0;

  const uint32_t idesc_b = make_idesc(NC, NB);
  const uint32_t idesc_c = make_idesc(NC, Kb);
  const uint32_t idesc_c2 = make_idesc(NC, 2 * Kb);
  const int lq = warp & 3, hb = warp >> 2;  // lane quarter of tensor memory, column half
  const int my_col = 32 * lq + lane;
  uint32_t phase = 0;
  for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
    const int k = tile / nst, s0 = (tile % nst) * ST, ns = min(ST, S - s0);
    const float* wvk = a.wv + (size_t)k * Nt * Np;
    const int tnext = tile + gridDim.x;
    const bool has_next = tnext < ntiles;
    const int kn = tnext / nst, s0n = (tnext % nst) * ST;
    for (int c0 = 0, ch = 0; ok && c0 < NP; c0 += RC, ++ch) {
      const bool last = c0 + RC >= NP;
      __syncthreads();  // the previous chunk's stage D is done with PT and AP
      if (ft >= 0) {
        float4* dst = reinterpret_cast<float4*>(PT);
        const int n4 = (RL + 4) * RC / 4;
  #pragma unroll
        for (int u = 0; u < kTaPtRegs; ++u) {
          const int i = u * kFetchThreads + ft;
          if (i < n4) dst[i] = pt_reg[u];
        }
  #pragma unroll
        for (int u = 0; u < kTaWvRegs; ++u) {
          const int i = u * kFetchThreads + ft;
          if (wv_pq[u] >= 0) WV[i] = wv_reg[u];
        }
      }
      __syncthreads();
      // ---- A: Legendre sums (4 pairs x 4 states per item) into the FP32 F rows [kap][col],
      //      kap = m + lmax
      {
        constexpr int NPB = RC / 4, NSB = ST / 4, NCMB = NPB * NSB;
        for (int it = tid; it < M2 * NCMB; it += kTaThreads) {
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
          // columns 16 p + 4 sp + 2 r + e: r = 0 row j (E + O), r = 1 mirror row jb (E - O)
          float* frow = F32 + (size_t)(m + lmax) * kNCp + 2 * s0l;
  #pragma unroll
          for (int u = 0; u < 4; ++u) {
            float* f = frow + (size_t)(p0 + u) * 16;
            st4(f, E[u][0] + O[u][0], E[u][1] + O[u][1], E[u][0] - O[u][0], E[u][1] - O[u][1]);
            st4(f + 4, E[u][2] + O[u][2], E[u][3] + O[u][3], E[u][2] - O[u][2], E[u][3] - O[u][3]);
          }
        }
      }
      __syncthreads();
      // F rows -> split BF16 F operand (row = column col, K = kap; kap >= M2 zero). Task = one
      // column and 8 consecutive kap: 8 lanes fill 128 contiguous bytes of each plane.
      for (int t = tid; t < NC * (Kb / 8); t += kTaThreads) {
        const int col = t & (NC - 1), k0 = (t >> 7) * 8;
        float x[8];
  #pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = (k0 + i < M2) ? F32[(size_t)(k0 + i) * kNCp + col] : 0.f;
        uint4 h, lo;
        split2(x[0], x[1], h.x, lo.x);
        split2(x[2], x[3], h.y, lo.y);
        split2(x[4], x[5], h.z, lo.z);
        split2(x[6], x[7], h.w, lo.w);
        const int off = canon_off(col, k0, NC);
        *reinterpret_cast<uint4*>(Fhi + off) = h;
        *reinterpret_cast<uint4*>(Flo + off) = lo;
      }
      // the tile's last stage A has read Gs: stream the next tile's G into it
      if (last && has_next) prefetch_g(kn, s0n);
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      // ---- B: grid values on all angles, D_B[col][p] (tensor memory columns 0 .. NB-1)
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_hi = smem_u32(Fhi), a_lo = smem_u32(Flo);
        const uint32_t b_hi = smem_u32(smem + sh.off_tb);
        const uint32_t b_lo = b_hi + (uint32_t)NB * Kb * 2;
        for (int ks = 0; ks < Kb / 16; ++ks) {
          const uint32_t ao = ks * (NC / 8) * 256, bo = ks * (NB / 8) * 256;
          const uint64_t dah = make_desc(a_hi + ao, 128, 256), dal = make_desc(a_lo + ao, 128, 256);
          const uint64_t dbh = make_desc(b_hi + bo, 128, 256), dbl = make_desc(b_lo + bo, 128, 256);
          mma_bf16(tmem, dah, dbh, idesc_b, ks > 0 ? 1u : 0u);
          mma_bf16(tmem, dah, dbl, idesc_b, 1u);
          mma_bf16(tmem, dal, dbh, idesc_b, 1u);
        }
        mma_commit(bar_mma);
      }
      // the next chunk's rows: their loads run while the MMAs and the later stages compute
      if (!last) fetch_chunk(wvk, c0 + RC, ch + 1);
      else if (has_next) fetch_chunk(a.wv + (size_t)kn * Nt * Np, 0, 0);
      bool w_ok = mbar_wait(bar_mma, phase);
      phase ^= 1u;
      if (!w_ok) atomicCAS(err, 0, 2);
      ok = __syncthreads_and(w_ok ? 1 : 0) != 0;
      if (!ok) break;
      tc_fence_after();
      // ---- W V on the grid; g = W V x D_B as split BF16 at (col, p) of the g operand. Warp:
      //      lane quarter lq (columns 32 lq ..), half hb of the angles.
      {
        const int col = my_col;
        const int pr = 2 * (col >> 4) + ((col >> 1) & 1);
        const float* wrow = WV + (size_t)pr * Np;
        const int half = NB / 2;
        const bool wv4 = (Np & 3) == 0;  // W V rows 16-byte aligned
        for (int pb0 = hb * half; pb0 < (hb + 1) * half; pb0 += 32) {
          float v[32];
          const uint32_t ta = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)pb0;
          tmem_ld16_issue(ta, v);
          tmem_ld16_issue(ta + 16, v + 16);
          tmem_ld_wait();
  #pragma unroll
          for (int o8 = 0; o8 < 4; ++o8) {
            const int p0 = pb0 + 8 * o8;
            float w[8];
            if (wv4 && p0 + 8 <= Np) {
              unpack4(ld4(wrow + p0), w);
              unpack4(ld4(wrow + p0 + 4), w + 4);
            } else {
  #pragma unroll
              for (int i = 0; i < 8; ++i) w[i] = (p0 + i < Np) ? wrow[p0 + i] : 0.f;
            }
            const float* vv = v + 8 * o8;
            uint4 h, lo;
            split2(vv[0] * w[0], vv[1] * w[1], h.x, lo.x);
            split2(vv[2] * w[2], vv[3] * w[3], h.y, lo.y);
            split2(vv[4] * w[4], vv[5] * w[5], h.z, lo.z);
            split2(vv[6] * w[6], vv[7] * w[7], h.w, lo.w);
            const int off = canon_off(col, p0, NC);
            *reinterpret_cast<uint4*>(Ghi + off) = h;
            *reinterpret_cast<uint4*>(Glo + off) = lo;
          }
        }
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      // ---- C: phi quadrature. The B operand stacks the hi rows of T^T over its lo rows, so one
      //      MMA of N = 2 Kb gives hi*hi (columns NB ..) and hi*lo (columns NB + Kb ..), and one of
      //      N = Kb adds lo*hi to the first block: D_C = sum of the two blocks.
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_hi = smem_u32(Ghi), a_lo = smem_u32(Glo);
        const uint32_t b = smem_u32(smem + sh.off_tc);
        for (int ks = 0; ks < NB / 16; ++ks) {
          const uint32_t ao = ks * (NC / 8) * 256, bo = ks * (2 * Kb / 8) * 256;
          const uint64_t dah = make_desc(a_hi + ao, 128, 256), dal = make_desc(a_lo + ao, 128, 256);
          const uint64_t db = make_desc(b + bo, 128, 256);
          mma_bf16(tmem + (uint32_t)NB, dah, db, idesc_c2, ks > 0 ? 1u : 0u);
          mma_bf16(tmem + (uint32_t)NB, dal, db, idesc_c, 1u);
        }
        mma_commit(bar_mma);
      }
      w_ok = mbar_wait(bar_mma, phase);
      phase ^= 1u;
      if (!w_ok) atomicCAS(err, 0, 3);
      ok = __syncthreads_and(w_ok ? 1 : 0) != 0;
      if (!ok) break;
      tc_fence_after();
      // ---- combine the mirror rows: AP[kap][p][0][s] = A_j + A_jb, AP[kap][p][1][s] = A_j - A_jb;
      //      the mirror of column col is col ^ 2 (lane ^ 2)
      {
        const int col = my_col;
        const int pp = col >> 4, r = (col >> 1) & 1, s = 2 * ((col >> 2) & 3) + (col & 1);
        const int half = Kb / 2;
        for (int kb0 = hb * half; kb0 < (hb + 1) * half; kb0 += 16) {
          float v[16], w[16];
          const uint32_t ta = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(NB + kb0);
          tmem_ld16_issue(ta, v);
          tmem_ld16_issue(ta + (uint32_t)Kb, w);
          tmem_ld_wait();
  #pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += w[i];
  #pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float other = __shfl_xor_sync(0xffffffffu, v[i], 2);
            const int kap = kb0 + i;
            if (kap < M2)
              AP[(size_t)kap * kAPS + (pp * 2 + r) * ST + s] = r ? other - v[i] : v[i] + other;
          }
        }
      }
      tc_fence_before();
      __syncthreads();
      // ---- D: Legendre quadrature into the item's register sums (rows past lmax read as zero)
      if (d_live) {
        float pv[kGmLq][RC];
  #pragma unroll
        for (int v = 0; v < kGmLq; ++v) {
          const int l = d_lbase + 2 * v;
          if (l <= lmax) {
            const float* prw = PT + (size_t)(theta_off(L, d_am) + l - d_am) * RC;
            unpack4(ld4(prw), pv[v]);
            unpack4(ld4(prw + 4), pv[v] + 4);
          } else {
  #pragma unroll
            for (int q = 0; q < RC; ++q) pv[v][q] = 0.f;
          }
        }
        const float* arow = AP + (size_t)d_mi * kAPS + (d_par ? ST : 0);
  #pragma unroll
        for (int pp = 0; pp < RC; ++pp) {
          float av[ST];
          unpack4(ld4(arow + (size_t)pp * 2 * ST), av);
          unpack4(ld4(arow + (size_t)pp * 2 * ST + 4), av + 4);
  #pragma unroll
          for (int v = 0; v < kGmLq; ++v)
  #pragma unroll
            for (int q = 0; q < ST; ++q) dacc[v][q] = fmaf(pv[v][pp], av[q], dacc[v][q]);
        }
      }
    }
    if (!ok) break;
    // the item's sums go straight to G (8 consecutive states of one (l, m) row), then reset
    if (d_live) {
      const bool vec = (S & 3) == 0 && ns == ST && (reinterpret_cast<uintptr_t>(G) & 15) == 0;
  #pragma unroll
      for (int v = 0; v < kGmLq; ++v) {
        const int l = d_lbase + 2 * v;
        if (l <= lmax) {
          float* gr = G + ((size_t)k * L2 + l * l + l + d_m) * S + s0;
          if (vec) {
            st4(gr, dacc[v][0], dacc[v][1], dacc[v][2], dacc[v][3]);
            st4(gr + 4, dacc[v][4], dacc[v][5], dacc[v][6], dacc[v][7]);
          } else {
  #pragma unroll
            for (int q = 0; q < ST; ++q)
              if (q < ns) gr[q] = dacc[v][q];
          }
        }
  #pragma unroll
        for (int q = 0; q < ST; ++q) dacc[v][q] = 0.f;
      }
    }
    cp_async_wait_all();
    __syncthreads();  // the next tile's Gs is complete
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

}  // namespace

bool angular_tc_eligible(int L, int n_theta, int n_phi) {
  const TaShape s = ta_shape(L, n_theta, n_phi);
  return s.NB <= 256 && 2 * s.Kb <= 256 && s.NB + 2 * s.Kb <= 512 && s.total <= 227 * 1024 &&
         L * L * kST <= kGmGRegs * kTaThreads && gm_items(L) <= kTaThreads &&
         (s.RL + 4) * kRC / 4 <= kTaPtRegs * kFetchThreads &&
         2 * kRC * n_phi <= kTaWvRegs * kFetchThreads && s.M2 <= 255;
}

bool angular_tc_enabled() {
  const char* e = getenv("CS_ANGULAR_KERNEL");
  return !e || (e[0] == 't' && e[1] == 'c');
}

void build_tc_phi_table(int L, int n_phi, std::vector<uint16_t>& out) {
  const TaShape s = ta_shape(L, 1, n_phi);
  const int lmax = L - 1;
  const size_t nb = (size_t)s.NB * s.Kb;
  out.assign(4 * nb, 0);
  uint16_t* tbh = out.data();
  uint16_t* tbl = tbh + nb;
  uint16_t* tc2 = tbl + nb;  // 2 Kb rows: hi, then lo
  auto bits = [](__nv_bfloat16 b) -> uint16_t { return *reinterpret_cast<uint16_t*>(&b); };
  for (int p = 0; p < n_phi; ++p)
    for (int kap = 0; kap < s.M2; ++kap) {
      const int m = kap - lmax, am = m < 0 ? -m : m;
      const double ang = 2.0 * 3.14159265358979323846 * (double)((long long)am * p % n_phi) / n_phi;
      double v = m >= 0 ? std::cos(ang) : std::sin(ang);
      if (std::fabs(v) < 1e-12) v = 0.0;
      const float f = (float)v;
      const __nv_bfloat16 hb = __float2bfloat16_rn(f);
      const __nv_bfloat16 lb = __float2bfloat16_rn(f - __bfloat162float(hb));
      const int ob = canon_off(p, kap, s.NB) / 2;
      tbh[ob] = bits(hb);
      tbl[ob] = bits(lb);
      tc2[canon_off(kap, p, 2 * s.Kb) / 2] = bits(hb);
      tc2[canon_off(s.Kb + kap, p, 2 * s.Kb) / 2] = bits(lb);
    }
}

cudaError_t launch_angular_tc(const AngArgs<float>& a, const void* tphi, float* G, int* err,
                              cudaStream_t stream) {
  if (!tphi || !a.theta_pairs || !angular_tc_eligible(a.L, a.n_theta, a.n_phi))
    return cudaErrorInvalidConfiguration;
  const TaShape s = ta_shape(a.L, a.n_theta, a.n_phi);
  cudaError_t e = cudaFuncSetAttribute(k_angular_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)s.total);
  if (e != cudaSuccess) return e;
  // SM count of the current device, looked up on every launch (no shared state)
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const int ntiles = ((a.S + kST - 1) / kST) * a.n_r;
  const int grid = ntiles < nsm ? ntiles : nsm;  // persistent: one CTA per SM
  k_angular_tc<<<grid, kTaThreads, s.total, stream>>>(
      a, static_cast<const __nv_bfloat16*>(tphi), G, err);
  return cudaGetLastError();
}

}  // namespace cs
