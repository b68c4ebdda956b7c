// Angular block of H.X (Sec. 2.2.2 eq. Ar_lm, the inverse transform of Sec. 2.2.4) for the
// mixed-precision filter, entirely on the 5th-generation tensor cores, for any lmax whose
// operands fit: three passes over an FP32 intermediate FA in device memory.
//
//   L1  (per m, tcgen05)  F[t][m][s] = sum_l Theta_lm(t) G[l,m][s]: for each mode m and each
//       parity of l - |m|, one product over l with the states as the MMA's 128 rows and the
//       theta pairs as its columns (E = even l - |m|, O = odd); the mirror rows follow from the
//       parity of the associated Legendre functions, F(t) = E + O, F(pi - t) = E - O.
//   P   (per grid row, tcgen05) the phi synthesis, the W V product and the phi quadrature of
//       one (radial node k, theta row t) with the states as rows. The uniform phi grid
//       (n_phi a multiple of 4) is folded onto its quarter q = 0 .. n_phi/4: the modes split
//       into four classes (cos with m even / m odd, sin with m even / m odd), each a dense
//       product with the class's trig table at the quarter angles, and the grid values at the
//       four mirror angles q, n/2 - q, n/2 + q, n - q are +- combinations of the four class
//       sums. The quadrature is the transposed fold (duplicate mirror angles at q = 0 and
//       q = n/4 counted once).
//   L2  (per m, tcgen05)  G'[l,m][s] = sum_t Theta_lm(t) AP[t][m][s], with the mirror rows
//       folded into even and odd parts first: the adjoint of L1.
// Every product is split BF16 (hi = bf16(x), lo = bf16(x - hi); hi*hi + hi*lo + lo*hi
// accumulated in FP32 tensor memory); the Legendre and trig operands are split at set-up
// and laid out in the canonical K-major no-swizzle layout, copied per CTA by the TMA engine
// (cp.async.bulk). The block's states are the MMA rows (at most 128 per block; larger sets
// run as several blocks). FA holds [block][k][t][kap][SW] floats (kap = m + lmax, SW the
// state stride): L1 writes F there, P replaces each row's F by its AP in place, L2 reads it.
// Every mbarrier wait is bounded: on expiry the kernel records an error code in a device
// word, releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "cs_internal.h"
#include "hx_kernels.cuh"
#include "tc_common.cuh"

namespace cs {

namespace {

using namespace tcx;

constexpr int kWaThreads = 256;
constexpr int kPThreads = 512;  // the phi pass
constexpr int kWaRows = 128;  // MMA M: the states of one block
constexpr int kSmemPerSM = 228 * 1024;

__host__ __device__ inline int r16(int x) { return (x + 15) & ~15; }

// kap of item i of phi class c: 0 cos m = 2i, 1 cos m = 2i + 1, 2 sin m = 2i + 2,
// 3 sin m = 2i + 1 (sin modes have m < 0); -1 past the class
__host__ __device__ inline int class_kap(int c, int i, int lmax) {
  const int m = (c == 0) ? 2 * i : (c == 2) ? 2 * i + 2 : 2 * i + 1;
  if (m > lmax) return -1;
  return c < 2 ? lmax + m : lmax - m;
}

struct WaShape {
  int L, lmax, M2, Nt, NP, Np, Q;
  int NPp, KL, QP, KC;  // padded: theta pairs, l per parity, quarter angles, modes per class
  size_t leg_per_a;     // bytes of one |m| block of a Legendre table (both parities, hi, lo)
  size_t off_u, off_phi, phi_bytes, total;  // table image offsets (bytes)
};

__host__ __device__ inline WaShape wa_shape(int L, int n_theta, int n_phi) {
  WaShape s;
  s.L = L;
  s.lmax = L - 1;
  s.M2 = 2 * L - 1;
  s.Nt = n_theta;
  s.NP = (n_theta + 1) / 2;
  s.Np = n_phi;
  s.Q = n_phi / 4;
  s.NPp = r16(s.NP);
  s.KL = r16((L + 1) / 2);
  s.QP = r16(s.Q + 1);
  s.KC = r16(s.lmax / 2 + 1);
  s.leg_per_a = (size_t)4 * s.NPp * s.KL * 2;
  s.off_u = (size_t)L * s.leg_per_a;
  s.off_phi = 2 * s.off_u;
  s.phi_bytes = (size_t)2 * 4 * 2 * s.QP * s.KC * 2;
  s.total = s.off_phi + s.phi_bytes;
  return s;
}

__host__ __device__ inline uint32_t pow2_cols(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// shared memory of the three kernels (bytes)
__host__ __device__ inline size_t l1_smem(const WaShape& s) {
  return (size_t)2 * 2 * kWaRows * s.KL * 2 + (size_t)s.leg_per_a;
}
__host__ __device__ inline size_t l2_smem(const WaShape& s) {
  return (size_t)2 * 2 * kWaRows * s.NPp * 2 + (size_t)s.leg_per_a;
}
// quarter angles per quadrature pass of the phi kernel
__host__ __device__ inline int p_qh(int QP) { return (QP % 32 == 0) ? 32 : 16; }
struct PSmem {
  size_t f, a, tab, wv, total;
};
__host__ __device__ inline PSmem p_smem(const WaShape& s, int SW) {
  PSmem p;
  size_t o = 0;
  p.tab = o;  // trig tables first (one bulk copy at the start)
  o += s.phi_bytes;
  p.a = o;    // F operand / folded grid-value operand (4 classes each)
  size_t ab = (size_t)4 * 2 * kWaRows * s.KC * 2;
  const size_t hb = (size_t)4 * 2 * kWaRows * p_qh(s.QP) * 2;
  if (hb > ab) ab = hb;
  o += ab;
  p.f = o;    // the row's F, [M2][SW] floats
  o += (size_t)s.M2 * SW * 4;
  p.wv = o;   // W V of the row, double buffered
  o += (size_t)2 * s.Np * 4;
  p.total = o;
  return p;
}

__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// 8 values at (row, k0 .. k0 + 7) of a split operand pair (hi plane, lo plane) of `rows` rows
__device__ __forceinline__ void store_split8(unsigned char* hi, unsigned char* lo, int row, int k0,
                                             int rows, const float* x) {
  uint4 h, l;
  split2(x[0], x[1], h.x, l.x);
  split2(x[2], x[3], h.y, l.y);
  split2(x[4], x[5], h.z, l.z);
  split2(x[6], x[7], h.w, l.w);
  const int off = canon_off(row, k0, rows);
  *reinterpret_cast<uint4*>(hi + off) = h;
  *reinterpret_cast<uint4*>(lo + off) = l;
}

// item it of the mode list (0: m = 0; 2a - 1: m = +a; 2a: m = -a)
__device__ __forceinline__ int item_m(int it) { return it == 0 ? 0 : ((it & 1) ? (it + 1) / 2 : -(it / 2)); }

struct WaArgs {
  int L, n_r, Nt, Np, S, SW, nblk, nmr;
  const float* wv;                // [k][t][p]
  const unsigned char* tab;       // set-up image (Legendre B, Legendre U, phi T and U)
  float* G;                       // [k][lm][S]
  float* FA;                      // [block][k][t][kap][SW]
  int* err;
};

__device__ __forceinline__ void record(int* err, int code) { atomicCAS(err, 0, code); }

// ------------------------------------------------------------------------------------ L1
// NT: operand tasks (8 values each) per thread and mode, an upper bound on KL / 8. The next
// mode's G values are loaded into registers while this mode's MMAs and stores run.
template <int NT>
__global__ void __launch_bounds__(kWaThreads)
    k_leg_synth_tc(WaArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_sh;
  const WaShape sh = wa_shape(a.L, a.Nt, a.Np);
  const int L = a.L, lmax = L - 1, L2 = L * L, M2 = sh.M2, KL = sh.KL, NPp = sh.NPp, NP = sh.NP;
  const int Nt = a.Nt, S = a.S, SW = a.SW;
  const int tile = blockIdx.x;
  const int r = tile % a.nmr, k = (tile / a.nmr) % a.n_r, blk = tile / (a.nmr * a.n_r);
  const int s0 = blk * kWaRows, ns = min(kWaRows, S - s0);
  const int it0 = (int)((long long)r * M2 / a.nmr), it1 = (int)((long long)(r + 1) * M2 / a.nmr);
  unsigned char* sA = smem;                                  // [par][hi|lo][128 x KL]
  unsigned char* sB = smem + (size_t)4 * kWaRows * KL * 2;   // [par][hi|lo][NPp x KL]
  const size_t aplane = (size_t)kWaRows * KL * 2, bplane = (size_t)NPp * KL * 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t bar_tab = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
  const uint32_t tcols = pow2_cols(2 * NPp);
  const int ntask = kWaRows * 2 * (KL / 8);
  if (tid == 0) {
    mbar_init(bar_tab, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_sh), tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t idesc = make_idesc(kWaRows, NPp);
  // A[par][s][i] = G[k][l = am + par + 2i, m][s0 + s] (zero past lmax and past the states)
  float gx[NT][8];
  auto load = [&](int it) {
    const int m = item_m(it), am = m < 0 ? -m : m;
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int task = tid + u * kWaThreads;
      const int s = task & (kWaRows - 1), rest = task >> 7;
      const int par = rest & 1, ig = rest >> 1;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int l = am + par + 2 * (8 * ig + j);
        gx[u][j] = (task < ntask && l <= lmax && s < ns)
                       ? a.G[((size_t)k * L2 + l * l + l + m) * S + s0 + s]
                       : 0.f;
      }
    }
  };
  if (it0 < it1) load(it0);
  uint32_t ph_tab = 0, ph_mma = 0;
  int cur_a = -1;
  bool ok = true;
  for (int it = it0; it < it1 && ok; ++it) {
    const int m = item_m(it), am = m < 0 ? -m : m, kap = m + lmax;
    const bool load_tab = am != cur_a;
    if (load_tab && tid == 0) {
      mbar_expect_tx(bar_tab, (uint32_t)sh.leg_per_a);
      bulk_g2s(smem_u32(sB), a.tab + (size_t)am * sh.leg_per_a, (uint32_t)sh.leg_per_a, bar_tab);
    }
    cur_a = am;
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int task = tid + u * kWaThreads;
      if (task < ntask) {
        const int s = task & (kWaRows - 1), rest = task >> 7;
        const int par = rest & 1, ig = rest >> 1;
        unsigned char* hi = sA + (size_t)par * 2 * aplane;
        store_split8(hi, hi + aplane, s, 8 * ig, kWaRows, gx[u]);
      }
    }
    if (it + 1 < it1) load(it + 1);
    fence_async_smem();
    tc_fence_before();
    bool t_ok = true;
    if (load_tab) {
      t_ok = mbar_wait(bar_tab, ph_tab);
      ph_tab ^= 1u;
      if (!t_ok) record(a.err, 21);
    }
    ok = __syncthreads_and(t_ok ? 1 : 0) != 0;
    if (!ok) break;
    if (tid == 0) {
      tc_fence_after();
      for (int par = 0; par < 2; ++par) {
        const uint32_t ah = smem_u32(sA + (size_t)par * 2 * aplane), al = ah + (uint32_t)aplane;
        const uint32_t bh = smem_u32(sB + (size_t)par * 2 * bplane), bl = bh + (uint32_t)bplane;
        for (int ks = 0; ks < KL / 16; ++ks) {
          const uint32_t ao = ks * (kWaRows / 8) * 256, bo = ks * (NPp / 8) * 256;
          const uint64_t dah = make_desc(ah + ao, 128, 256), dal = make_desc(al + ao, 128, 256);
          const uint64_t dbh = make_desc(bh + bo, 128, 256), dbl = make_desc(bl + bo, 128, 256);
          const uint32_t d = tmem + (uint32_t)(par * NPp);
          mma_bf16(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
          mma_bf16(d, dah, dbl, idesc, 1u);
          mma_bf16(d, dal, dbh, idesc, 1u);
        }
      }
      mma_commit(bar_mma);
    }
    const bool w_ok = mbar_wait(bar_mma, ph_mma);
    ph_mma ^= 1u;
    if (!w_ok) record(a.err, 22);
    ok = __syncthreads_and(w_ok ? 1 : 0) != 0;
    if (!ok) break;
    tc_fence_after();
    // F(t) = E + O, F(mirror t) = E - O for this warp's lane quarter (states), every other
    // 16 pairs
    {
      const int qd = warp & 3, hh = warp >> 2, s = 32 * qd + lane;
      float* base = a.FA + (((size_t)blk * a.n_r + k) * Nt) * (size_t)M2 * SW;
      for (int t0 = 16 * hh; t0 < NPp; t0 += 32) {
        float e[16], o[16];
        const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)t0;
        tmem_ld16_issue(ta, e);
        tmem_ld16_issue(ta + (uint32_t)NPp, o);
        tmem_ld_wait();
        if (s < SW) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int t = t0 + j;
            if (t < NP) {
              const int tb = Nt - 1 - t;
              base[((size_t)t * M2 + kap) * SW + s] = e[j] + o[j];
              if (tb != t) base[((size_t)tb * M2 + kap) * SW + s] = e[j] - o[j];
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------------------------------------------ L2
// 512 threads. NT: operand tasks (8 pairs each) per thread and mode, an upper bound on NPp / 32;
// the next
// mode's AP values are loaded into registers while this mode's MMAs and stores run.
template <int NT>
__global__ void __launch_bounds__(kPThreads, 1)
    k_leg_anal_tc(WaArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_sh;
  const WaShape sh = wa_shape(a.L, a.Nt, a.Np);
  const int L = a.L, lmax = L - 1, L2 = L * L, M2 = sh.M2, KL = sh.KL, NPp = sh.NPp, NP = sh.NP;
  const int Nt = a.Nt, S = a.S, SW = a.SW;
  const int tile = blockIdx.x;
  const int r = tile % a.nmr, k = (tile / a.nmr) % a.n_r, blk = tile / (a.nmr * a.n_r);
  const int s0 = blk * kWaRows, ns = min(kWaRows, S - s0);
  const int it0 = (int)((long long)r * M2 / a.nmr), it1 = (int)((long long)(r + 1) * M2 / a.nmr);
  unsigned char* sA = smem;                                   // [par][hi|lo][128 x NPp]
  unsigned char* sU = smem + (size_t)4 * kWaRows * NPp * 2;   // [par][hi|lo][KL x NPp]
  const size_t aplane = (size_t)kWaRows * NPp * 2, uplane = (size_t)KL * NPp * 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t bar_tab = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
  const uint32_t tcols = pow2_cols(2 * KL);
  const int ntask = kWaRows * (NPp / 8);
  if (tid == 0) {
    mbar_init(bar_tab, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_sh), tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const uint32_t idesc = make_idesc(kWaRows, KL);
  const float* base = a.FA + (((size_t)blk * a.n_r + k) * Nt) * (size_t)M2 * SW;
  // AP(t) and AP(mirror t) of the task's 8 pairs (the self-mirror row of an odd n_theta has
  // no mirror: its second value stays zero and it enters the even part only)
  float xv[NT][8], yv[NT][8];
  auto load = [&](int it) {
    const int kap = item_m(it) + lmax;
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int task = tid + u * kPThreads;
      const int s = task & (kWaRows - 1), tg = task >> 7;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int t = 8 * tg + j, tb = Nt - 1 - t;
        const bool in = task < ntask && t < NP && s < SW;
        xv[u][j] = in ? base[((size_t)t * M2 + kap) * SW + s] : 0.f;
        yv[u][j] = (in && tb != t) ? base[((size_t)tb * M2 + kap) * SW + s] : 0.f;
      }
    }
  };
  if (it0 < it1) load(it0);
  uint32_t ph_tab = 0, ph_mma = 0;
  int cur_a = -1;
  bool ok = true;
  for (int it = it0; it < it1 && ok; ++it) {
    const int m = item_m(it), am = m < 0 ? -m : m;
    const bool load_tab = am != cur_a;
    if (load_tab && tid == 0) {
      mbar_expect_tx(bar_tab, (uint32_t)sh.leg_per_a);
      bulk_g2s(smem_u32(sU), a.tab + sh.off_u + (size_t)am * sh.leg_per_a,
               (uint32_t)sh.leg_per_a, bar_tab);
    }
    cur_a = am;
    // A[0][s][t] = AP(t) + AP(mirror t), A[1][s][t] = AP(t) - AP(mirror t)
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int task = tid + u * kPThreads;
      if (task < ntask) {
        const int s = task & (kWaRows - 1), tg = task >> 7;
        float e[8], o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int t = 8 * tg + j;
          e[j] = xv[u][j] + yv[u][j];
          o[j] = (Nt - 1 - t != t) ? xv[u][j] - yv[u][j] : 0.f;
        }
        store_split8(sA, sA + aplane, s, 8 * tg, kWaRows, e);
        store_split8(sA + 2 * aplane, sA + 3 * aplane, s, 8 * tg, kWaRows, o);
      }
    }
    if (it + 1 < it1) load(it + 1);
    fence_async_smem();
    tc_fence_before();
    bool t_ok = true;
    if (load_tab) {
      t_ok = mbar_wait(bar_tab, ph_tab);
      ph_tab ^= 1u;
      if (!t_ok) record(a.err, 23);
    }
    ok = __syncthreads_and(t_ok ? 1 : 0) != 0;
    if (!ok) break;
    if (tid == 0) {
      tc_fence_after();
      for (int par = 0; par < 2; ++par) {
        const uint32_t ah = smem_u32(sA + (size_t)par * 2 * aplane), al = ah + (uint32_t)aplane;
        const uint32_t uh = smem_u32(sU + (size_t)par * 2 * uplane), ul = uh + (uint32_t)uplane;
        for (int ks = 0; ks < NPp / 16; ++ks) {
          const uint32_t ao = ks * (kWaRows / 8) * 256, uo = ks * (KL / 8) * 256;
          const uint64_t dah = make_desc(ah + ao, 128, 256), dal = make_desc(al + ao, 128, 256);
          const uint64_t duh = make_desc(uh + uo, 128, 256), dul = make_desc(ul + uo, 128, 256);
          const uint32_t d = tmem + (uint32_t)(par * KL);
          mma_bf16(d, dah, duh, idesc, ks > 0 ? 1u : 0u);
          mma_bf16(d, dah, dul, idesc, 1u);
          mma_bf16(d, dal, duh, idesc, 1u);
        }
      }
      mma_commit(bar_mma);
    }
    const bool w_ok = mbar_wait(bar_mma, ph_mma);
    ph_mma ^= 1u;
    if (!w_ok) record(a.err, 24);
    ok = __syncthreads_and(w_ok ? 1 : 0) != 0;
    if (!ok) break;
    tc_fence_after();
    // G'[l = am + par + 2i, m][s]; warps 4..7 and 12..15 the odd parity, warps 8..15 every
    // other 16 l
    {
      const int qd = warp & 3, par = (warp >> 2) & 1, s = 32 * qd + lane;
      for (int i0 = 16 * (warp >> 3); i0 < KL; i0 += 32) {
        float v[16];
        tmem_ld16_issue(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(par * KL + i0), v);
        tmem_ld_wait();
        if (s < ns) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int l = am + par + 2 * (i0 + j);
            if (l <= lmax) a.G[((size_t)k * L2 + l * l + l + m) * S + s0 + s] = v[j];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

// ------------------------------------------------------------------------------------- P
// One tile = (block, k, t), 512 threads. Tensor-memory columns: synthesis class c at c QP
// (4 QP in all), quadrature class c at 4 QP + c KC. The quadrature runs in passes over QH
// quarter angles: each pass forms the four classes' folded grid values for its angles once,
// and its MMAs accumulate into the quadrature columns.
__global__ void __launch_bounds__(kPThreads, 1)
    k_phi_tc(WaArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[3];
  __shared__ uint32_t tmem_sh;
  const WaShape sh = wa_shape(a.L, a.Nt, a.Np);
  const int lmax = a.L - 1, M2 = sh.M2, KC = sh.KC, QP = sh.QP, Q = sh.Q, QH = p_qh(QP);
  const int Nt = a.Nt, Np = a.Np, SW = a.SW;
  const PSmem ps = p_smem(sh, SW);
  unsigned char* sT = smem + ps.tab;                       // [c][hi|lo][QP x KC]
  unsigned char* sUt = sT + (size_t)4 * 2 * QP * KC * 2;   // [c][hi|lo][KC x QP]
  unsigned char* sA = smem + ps.a;
  const float* Fst = reinterpret_cast<const float*>(smem + ps.f);
  const float* WVb = reinterpret_cast<const float*>(smem + ps.wv);
  const size_t fplane = (size_t)kWaRows * KC * 2, hplane = (size_t)kWaRows * QH * 2;
  const size_t tplane = (size_t)QP * KC * 2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t bar_tab = smem_u32(&bars[0]), bar_f = smem_u32(&bars[1]),
                 bar_mma = smem_u32(&bars[2]);
  const uint32_t tcols = pow2_cols(4 * QP + 4 * KC);
  const long long ntiles = (long long)a.nblk * a.n_r * Nt;
  const uint32_t fbytes = (uint32_t)((size_t)M2 * SW * 4), wbytes = (uint32_t)(Np * 4);
  if (tid == 0) {
    mbar_init(bar_tab, 1);
    mbar_init(bar_f, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_sh), tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_sh;
  // tile -> its FA row and W V row
  auto tile_src = [&](long long tl, const float*& f, const float*& w) {
    const int t = (int)(tl % Nt);
    const int k = (int)((tl / Nt) % a.n_r);  // tl / Nt = block n_r + k
    f = a.FA + (size_t)tl * M2 * SW;
    w = a.wv + ((size_t)k * Nt + t) * Np;
  };
  if (tid == 0) {
    mbar_expect_tx(bar_tab, (uint32_t)sh.phi_bytes);
    bulk_g2s(smem_u32(sT), a.tab + sh.off_phi, (uint32_t)sh.phi_bytes, bar_tab);
    if ((long long)blockIdx.x < ntiles) {
      const float *f, *w;
      tile_src(blockIdx.x, f, w);
      mbar_expect_tx(bar_f, fbytes + wbytes);
      bulk_g2s(smem_u32(smem + ps.f), f, fbytes, bar_f);
      bulk_g2s(smem_u32(smem + ps.wv), w, wbytes, bar_f);
    }
  }
  bool ok = mbar_wait(bar_tab, 0);
  if (!ok) record(a.err, 25);
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  const uint32_t idesc_s = make_idesc(kWaRows, QP), idesc_a = make_idesc(kWaRows, KC);
  const int qd = warp & 3, cg = warp >> 2, s_me = 32 * qd + lane;
  const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
  const int npass = QP / QH;
  uint32_t ph_f = 0, ph_mma = 0;
  int buf = 0;
  for (long long tl = blockIdx.x; ok && tl < ntiles; tl += gridDim.x, buf ^= 1) {
    bool w_ok = mbar_wait(bar_f, ph_f);
    ph_f ^= 1u;
    if (!w_ok) record(a.err, 26);
    ok = __syncthreads_and(w_ok ? 1 : 0) != 0;
    if (!ok) break;
    // ---- F operand of the four classes: A_c[s][i] = F[kap(c, i)][s]
    {
      const int ntask = kWaRows * 4 * (KC / 8);
      for (int task = tid; task < ntask; task += kPThreads) {
        const int s = task & (kWaRows - 1), rest = task >> 7;
        const int c = rest & 3, ig = rest >> 2;
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int kap = class_kap(c, 8 * ig + j, lmax);
          x[j] = (kap >= 0 && s < SW) ? Fst[(size_t)kap * SW + s] : 0.f;
        }
        unsigned char* hi = sA + (size_t)c * 2 * fplane;
        store_split8(hi, hi + fplane, s, 8 * ig, kWaRows, x);
      }
    }
    // the W V row of this tile stays in buffer `buf`; the next tile's goes to the other
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      const long long tn = tl + gridDim.x;
      if (tn < ntiles) {  // the F rows are consumed: stream the next tile's into them
        const float *f, *w;
        tile_src(tn, f, w);
        mbar_expect_tx(bar_f, fbytes + wbytes);
        bulk_g2s(smem_u32(smem + ps.f), f, fbytes, bar_f);
        bulk_g2s(smem_u32(smem + ps.wv + (size_t)(buf ^ 1) * Np * 4), w, wbytes, bar_f);
      }
      tc_fence_after();
      for (int c = 0; c < 4; ++c) {
        const uint32_t ah = smem_u32(sA + (size_t)c * 2 * fplane), al = ah + (uint32_t)fplane;
        const uint32_t bh = smem_u32(sT + (size_t)c * 2 * tplane), bl = bh + (uint32_t)tplane;
        for (int ks = 0; ks < KC / 16; ++ks) {
          const uint32_t ao = ks * (kWaRows / 8) * 256, bo = ks * (QP / 8) * 256;
          const uint64_t dah = make_desc(ah + ao, 128, 256), dal = make_desc(al + ao, 128, 256);
          const uint64_t dbh = make_desc(bh + bo, 128, 256), dbl = make_desc(bl + bo, 128, 256);
          const uint32_t d = tmem + (uint32_t)(c * QP);
          mma_bf16(d, dah, dbh, idesc_s, ks > 0 ? 1u : 0u);
          mma_bf16(d, dah, dbl, idesc_s, 1u);
          mma_bf16(d, dal, dbh, idesc_s, 1u);
        }
      }
      mma_commit(bar_mma);
    }
    w_ok = mbar_wait(bar_mma, ph_mma);
    ph_mma ^= 1u;
    if (!w_ok) record(a.err, 27);
    ok = __syncthreads_and(w_ok ? 1 : 0) != 0;
    if (!ok) break;
    tc_fence_after();
    const float* wvr = WVb + (size_t)buf * Np;
    for (int pass = 0; pass < npass && ok; ++pass) {
      // grid values at the four mirror angles of 8 quarter angles, times W V, folded back
      // into the four classes: h_c[s][q - pass QH]
      if (8 * cg < QH) {
        const int qc = pass * QH + 8 * cg;
        float v[4][8];
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem_ld8_issue(tmem + lane_base + (uint32_t)(c * QP + qc), v[c]);
        tmem_ld_wait();
        float h[4][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int q = qc + j;
          const float ce = v[0][j], co = v[1][j], se = v[2][j], so = v[3][j];
          float g1 = 0.f, g2 = 0.f, g3 = 0.f, g4 = 0.f;
          if (q <= Q) {
            const int p2 = 2 * Q - q, p3 = 2 * Q + q, p4 = 4 * Q - q;
            g1 = wvr[q] * (ce + co + se + so);
            if (q != Q) g2 = wvr[p2] * (ce - co - se + so);
            if (q != 0) g3 = wvr[p3] * (ce - co + se - so);
            if (q != 0 && q != Q) g4 = wvr[p4] * (ce + co - se - so);
          }
          h[0][j] = (g1 + g2) + (g3 + g4);
          h[1][j] = (g1 - g2) - (g3 - g4);
          h[2][j] = (g1 - g2) + (g3 - g4);
          h[3][j] = (g1 + g2) - (g3 + g4);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          unsigned char* hi = sA + (size_t)c * 2 * hplane;
          store_split8(hi, hi + hplane, s_me, 8 * cg, kWaRows, h[c]);
        }
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        for (int c = 0; c < 4; ++c) {
          const uint32_t ah = smem_u32(sA + (size_t)c * 2 * hplane), al = ah + (uint32_t)hplane;
          const uint32_t uh = smem_u32(sUt + (size_t)c * 2 * tplane), ul = uh + (uint32_t)tplane;
          for (int ks = 0; ks < QH / 16; ++ks) {
            const uint32_t ao = ks * (kWaRows / 8) * 256;
            const uint32_t uo = (pass * (QH / 16) + ks) * (KC / 8) * 256;
            const uint64_t dah = make_desc(ah + ao, 128, 256), dal = make_desc(al + ao, 128, 256);
            const uint64_t duh = make_desc(uh + uo, 128, 256), dul = make_desc(ul + uo, 128, 256);
            const uint32_t d = tmem + (uint32_t)(4 * QP + c * KC);
            mma_bf16(d, dah, duh, idesc_a, (pass > 0 || ks > 0) ? 1u : 0u);
            mma_bf16(d, dah, dul, idesc_a, 1u);
            mma_bf16(d, dal, duh, idesc_a, 1u);
          }
        }
        mma_commit(bar_mma);
      }
      w_ok = mbar_wait(bar_mma, ph_mma);
      ph_mma ^= 1u;
      if (!w_ok) record(a.err, 28);
      ok = __syncthreads_and(w_ok ? 1 : 0) != 0;
      tc_fence_after();
    }
    if (!ok) break;
    // AP[kap][s] in place of the row's F; warp column group cg writes class cg
    {
      float* dst = a.FA + (size_t)tl * M2 * SW;
      const int c = cg;
      for (int i0 = 0; i0 < KC; i0 += 16) {
        float v[16];
        tmem_ld16_issue(tmem + lane_base + (uint32_t)(4 * QP + c * KC + i0), v);
        tmem_ld_wait();
        if (s_me < SW) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int kap = class_kap(c, i0 + j, lmax);
            if (kap >= 0) dst[(size_t)kap * SW + s_me] = v[j];
          }
        }
      }
    }
    tc_fence_before();
  }
  // a bulk copy issued for a tile this CTA did not reach (error exit) must land before exit
  if (!ok && tid == 0) mbar_wait(bar_f, ph_f);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tcols);
}

// CTAs per SM that both shared memory and the tensor-memory columns allow; the dynamic
// shared memory request is raised so that no more than that many become resident
void residency(size_t smem, uint32_t tcols, int& per_sm, size_t& request) {
  const int by_tmem = (int)(512 / tcols);
  int by_smem = (int)(kSmemPerSM / (smem + 1024));
  if (by_smem < 1) by_smem = 1;
  per_sm = by_tmem < by_smem ? by_tmem : by_smem;
  request = smem;
  const size_t floor_req = (size_t)kSmemPerSM / (per_sm + 1) + 1;  // (per_sm + 1) do not fit
  if (request < floor_req) request = floor_req;
  if (request > 227 * 1024) request = 227 * 1024;
}

}  // namespace

bool angular_wide_eligible(int L, int n_theta, int n_phi) {
  if (L < 1 || n_theta < 2 || n_phi < 8 || (n_phi & 3) != 0) return false;
  const WaShape s = wa_shape(L, n_theta, n_phi);
  // register-prefetch bounds of the Legendre passes: KL <= 32 (lmax <= 62), NPp <= 64
  // (n_theta <= 128)
  if (s.NPp > 64 || s.KL > 32 || s.QP > 128 || s.KC > 128) return false;
  if (4 * s.QP + 4 * s.KC > 512 || 2 * s.NPp > 512) return false;
  if (l1_smem(s) > 200 * 1024 || l2_smem(s) > 200 * 1024) return false;
  return p_smem(s, kWaRows).total <= 220 * 1024;
}

bool angular_wide_enabled(int L, int n_theta, int n_phi, bool fused_eligible) {
  if (!angular_wide_eligible(L, n_theta, n_phi)) return false;
  const char* e = getenv("CS_ANGULAR_KERNEL");
  if (e && e[0] == 'w') return true;   // "wide"
  if (e && e[0] != '\0') return false;  // "tc" (fused) or "simt"
  return !fused_eligible;
}

int angular_wide_state_stride(int S) { return S >= kWaRows ? kWaRows : r16(S); }

size_t angular_wide_work_bytes(int L, int n_r, int n_theta, int S) {
  if (S <= 0) return 0;
  const int nblk = (S + kWaRows - 1) / kWaRows;
  return (size_t)nblk * n_r * n_theta * (2 * L - 1) * angular_wide_state_stride(S) * 4;
}

void build_wide_tables(const HostTables& H, std::vector<uint16_t>& out) {
  const WaShape s = wa_shape(H.L, H.n_theta, H.n_phi);
  out.assign(s.total / 2, 0);
  const int L = H.L, lmax = L - 1, rowlen = theta_row_len(L);
  auto bits = [](__nv_bfloat16 b) -> uint16_t { return *reinterpret_cast<uint16_t*>(&b); };
  auto put = [&](size_t plane_hi, size_t plane_lo, int row, int k, int rows, double v) {
    const float f = (float)v;
    const __nv_bfloat16 hb = __float2bfloat16_rn(f);
    const __nv_bfloat16 lb = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hb)));
    const size_t o = (size_t)canon_off(row, k, rows) / 2;
    out[plane_hi / 2 + o] = bits(hb);
    out[plane_lo / 2 + o] = bits(lb);
  };
  const size_t bpl = (size_t)s.NPp * s.KL * 2;  // bytes of one plane of a Legendre block
  for (int am = 0; am < L; ++am)
    for (int par = 0; par < 2; ++par)
      for (int i = 0; i < s.KL; ++i) {
        const int l = am + par + 2 * i;
        if (l > lmax) continue;
        for (int t = 0; t < s.NP; ++t) {
          const double v = H.theta[(size_t)t * rowlen + theta_off(L, am) + (l - am)];
          // L1's B operand: rows t, K = i
          const size_t b0 = (size_t)am * s.leg_per_a + (size_t)par * 2 * bpl;
          put(b0, b0 + bpl, t, i, s.NPp, v);
          // L2's B operand: rows i, K = t
          const size_t u0 = s.off_u + (size_t)am * s.leg_per_a + (size_t)par * 2 * bpl;
          put(u0, u0 + bpl, i, t, s.KL, v);
        }
      }
  const size_t tpl = (size_t)s.QP * s.KC * 2;
  const size_t uoff = s.off_phi + (size_t)4 * 2 * tpl;
  for (int c = 0; c < 4; ++c)
    for (int i = 0; i < s.KC; ++i) {
      if (class_kap(c, i, lmax) < 0) continue;
      const int m = (c == 0) ? 2 * i : (c == 2) ? 2 * i + 2 : 2 * i + 1;
      for (int q = 0; q <= s.Q; ++q) {
        const double ang =
            2.0 * 3.14159265358979323846 * (double)((long long)m * q % H.n_phi) / H.n_phi;
        double v = c < 2 ? std::cos(ang) : std::sin(ang);
        if (std::fabs(v) < 1e-12) v = 0.0;
        const size_t t0 = s.off_phi + (size_t)c * 2 * tpl;
        put(t0, t0 + tpl, q, i, s.QP, v);  // synthesis: rows q, K = i
        const size_t u0 = uoff + (size_t)c * 2 * tpl;
        put(u0, u0 + tpl, i, q, s.KC, v);  // quadrature: rows i, K = q
      }
    }
}

cudaError_t launch_angular_wide(const AngArgs<float>& a, const void* tab, float* G, float* FA,
                                int* err, cudaStream_t stream) {
  if (!tab || !FA || !angular_wide_eligible(a.L, a.n_theta, a.n_phi) || a.S <= 0)
    return cudaErrorInvalidConfiguration;
  const WaShape s = wa_shape(a.L, a.n_theta, a.n_phi);
  WaArgs w;
  w.L = a.L;
  w.n_r = a.n_r;
  w.Nt = a.n_theta;
  w.Np = a.n_phi;
  w.S = a.S;
  w.SW = angular_wide_state_stride(a.S);
  w.nblk = (a.S + kWaRows - 1) / kWaRows;
  w.wv = a.wv;
  w.tab = static_cast<const unsigned char*>(tab);
  w.G = G;
  w.FA = FA;
  w.err = err;
  cudaError_t e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  // Legendre passes: one CTA per (block, k, range of modes), about 6 CTAs per SM in all
  const int base = w.nblk * a.n_r;
  int nmr = (6 * nsm + base - 1) / base;
  // CS_WIDE_CTAS_PER_SM overrides the 6 CTAs per SM of the Legendre passes (for tuning)
  if (const char* e6 = getenv("CS_WIDE_CTAS_PER_SM")) {
    const int v = atoi(e6);
    if (v > 0 && v <= 64) nmr = (v * nsm + base - 1) / base;
  }
  if (nmr < 1) nmr = 1;
  if (nmr > s.M2) nmr = s.M2;
  w.nmr = nmr;
  int per_sm;
  size_t req;
  residency(l1_smem(s), pow2_cols(2 * s.NPp), per_sm, req);
  auto l1 = s.KL <= 16 ? k_leg_synth_tc<2> : k_leg_synth_tc<4>;
  if ((e = cudaFuncSetAttribute(l1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)req)) !=
      cudaSuccess)
    return e;
  l1<<<base * nmr, kWaThreads, req, stream>>>(w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const PSmem ps = p_smem(s, w.SW);
  residency(ps.total, pow2_cols(4 * s.QP + 4 * s.KC), per_sm, req);
  if ((e = cudaFuncSetAttribute(k_phi_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)req)) != cudaSuccess)
    return e;
  const long long ntiles = (long long)w.nblk * a.n_r * a.n_theta;
  long long grid = (long long)nsm * per_sm;
  if (grid > ntiles) grid = ntiles;
  k_phi_tc<<<(int)grid, kPThreads, req, stream>>>(w);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  residency(l2_smem(s), pow2_cols(2 * s.KL), per_sm, req);
  auto l2 = s.NPp <= 32 ? k_leg_anal_tc<1> : k_leg_anal_tc<2>;
  if ((e = cudaFuncSetAttribute(l2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)req)) !=
      cudaSuccess)
    return e;
  l2<<<base * nmr, kPThreads, req, stream>>>(w);
  return cudaGetLastError();
}

}  // namespace cs
