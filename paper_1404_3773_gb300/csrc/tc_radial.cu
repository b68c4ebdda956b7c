// Per-l radial contractions of H.X (Sec. 2.2.2 eqs. G_lmr and Arlm_to_coeff) on the 5th-
// generation tensor cores (tcgen05, sm_103a), for the mixed-precision filter:
//   synthesis : G_l[k][(m,s)]  = sum_n R_ln(r_k) X[alpha(l,m,n), s]      (M = k, K = n)
//   analysis  : Z[alpha(l,m,n), s] = sum_k R_ln(r_k) G'_l[k][(m,s)]       (M = n, K = k)
// Operands are BF16 in the canonical K-major no-swizzle layout (8-row x 16-byte core
// matrices). Each FP32 operand is split into hi = bf16(x) and lo = bf16(x - hi); the
// product is accumulated in FP32 tensor memory as hi*hi + hi*lo + lo*hi (split BF16), so
// the contraction keeps about 16 significant bits instead of 8.
// The radial tables are pre-split and pre-laid-out at set-up and copied to shared memory
// with cp.async.bulk (TMA engine) per K chunk; the state-side operand is converted while it
// is staged. One thread issues tcgen05.mma; completion is signalled through an mbarrier
// (tcgen05.commit); four warps read the accumulator back with tcgen05.ld (warp w owns
// TMEM lanes 32w .. 32w+31 = output rows) and run the epilogue of hx_kernels.cuh.
// Every mbarrier wait is bounded: on expiry the kernel records an error code in a device
// word, still waits (bounded) for its own MMAs, releases its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cs_internal.h"
#include "hx_kernels.cuh"
#include "tc_common.cuh"

namespace cs {

namespace {

constexpr int TM = 128;   // MMA M (output rows per tile)
constexpr int TN = 128;   // MMA N (output columns per tile) = TMEM columns allocated
constexpr int KC = 64;    // K elements per shared-memory chunk (4 MMA K-steps of 16)
constexpr int kThreads = 128;

using namespace tcx;

__host__ __device__ constexpr int chunk_bytes(int rows) { return rows * KC * 2; }

struct TcShape {
  int L, N, n_r, S;
  int m_tiles;   // output-row tiles of TM
  int kpad;      // K rounded up to KC
};

__device__ __forceinline__ void locate_tile(int tile, int S, int& l, int& c0) {
  l = 0;
  for (;;) {
    int ct = ((2 * l + 1) * S + TN - 1) / TN;
    if (tile < ct) break;
    tile -= ct;
    ++l;
  }
  c0 = tile * TN;
}

// MODE 0: synthesis (B from X, output G); MODE 1: analysis (B from G, epilogue to X layout)
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_tc_radial(TcShape sh,
                                                         const __nv_bfloat16* __restrict__ tab,
                                                         const float* __restrict__ X,
                                                         long long ldx, float* __restrict__ G,
                                                         Epilogue<float> ep,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];  // 4 x TM x KC bf16 = 64 KB
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base_sh;
  __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Alo = Ahi + TM * KC;
  __nv_bfloat16* Bhi = Alo + TM * KC;
  __nv_bfloat16* Blo = Bhi + TN * KC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int l, c0;
  locate_tile(blockIdx.x, sh.S, l, c0);
  const int mt = blockIdx.y;
  const int ncol = (2 * l + 1) * sh.S;
  const int L2 = sh.L * sh.L;
  const int Kdim = (MODE == 0) ? sh.N : sh.n_r;     // true K
  const int Mdim = (MODE == 0) ? sh.n_r : sh.N;     // true M
  const uint32_t bar_tma = smem_u32(&bars[0]);
  const uint32_t bar_mma = smem_u32(&bars[1]);
  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base_sh), TN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = tmem_base_sh;
  constexpr uint32_t idesc = make_idesc(TM, TN);
  bool ok = true;
  uint32_t phase = 0;
  // table layout: [l][m_tile][k chunk][hi|lo][TM x KC canonical]
  const int nchunks = sh.kpad / KC;
  const __nv_bfloat16* tab_l =
      tab + ((size_t)(l * sh.m_tiles + mt) * nchunks) * 2 * TM * KC;

  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int kb = ch * KC;
    if (tid == 0) {
      mbar_expect_tx(bar_tma, 2 * chunk_bytes(TM));
      bulk_g2s(smem_u32(Ahi), tab_l + (size_t)ch * 2 * TM * KC, 2 * chunk_bytes(TM), bar_tma);
    }
    // stage B (TN rows = output columns, KC K-elements) as split BF16
    if (MODE == 0) {
      // B[c][n] = X[(l^2 + mi) N + n + s ldx]; task = (column, octet of n)
      for (int t = tid; t < TN * (KC / 8); t += kThreads) {
        const int oc = t % (KC / 8), cc = t / (KC / 8);
        const int c = c0 + cc, n0 = kb + oc * 8;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.f;
        if (c < ncol) {
          const int mi = c / sh.S, s = c - mi * sh.S;
          const float* src = X + (size_t)(l * l + mi) * sh.N + (size_t)s * ldx;
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (n0 + i < Kdim) v[i] = src[n0 + i];
        }
        __align__(16) __nv_bfloat16 h[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split_bf16(v[i], h[i], lo[i]);
        const int off = canon_off(cc, oc * 8, TN);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Bhi) + off) =
            *reinterpret_cast<uint4*>(h);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Blo) + off) =
            *reinterpret_cast<uint4*>(lo);
      }
    } else {
      // B[c][k] = G[(k L^2 + l^2) S + c]; lanes over columns, loop over the k octet
      for (int t = tid; t < TN * (KC / 8); t += kThreads) {
        const int cc = t % TN, oc = t / TN;
        const int c = c0 + cc, k0 = kb + oc * 8;
        __align__(16) __nv_bfloat16 h[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float x = 0.f;
          if (c < ncol && k0 + i < Kdim) x = G[((size_t)(k0 + i) * L2 + l * l) * sh.S + c];
          split_bf16(x, h[i], lo[i]);
        }
        const int off = canon_off(cc, oc * 8, TN);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Bhi) + off) =
            *reinterpret_cast<uint4*>(h);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Blo) + off) =
            *reinterpret_cast<uint4*>(lo);
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(bar_tma, phase)) {
        atomicCAS(err, 0, 1);
        ok = false;
      } else {
        tc_fence_after();
        const uint32_t a_hi = smem_u32(Ahi), a_lo = smem_u32(Alo);
        const uint32_t b_hi = smem_u32(Bhi), b_lo = smem_u32(Blo);
#pragma unroll
        for (int ks = 0; ks < KC / 16; ++ks) {
          const uint32_t ao = ks * (TM / 8) * 256, bo = ks * (TN / 8) * 256;
          const uint64_t dah = make_desc(a_hi + ao, 128, 256), dal = make_desc(a_lo + ao, 128, 256);
          const uint64_t dbh = make_desc(b_hi + bo, 128, 256), dbl = make_desc(b_lo + bo, 128, 256);
          mma_bf16(tmem_d, dah, dbh, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
          mma_bf16(tmem_d, dah, dbl, idesc, 1u);
          mma_bf16(tmem_d, dal, dbh, idesc, 1u);
        }
      }
      mma_commit(bar_mma);  // arrives once the issued MMAs (if any) completed
    }
    // everyone waits for the MMAs of this chunk before the buffers are refilled
    if (!mbar_wait(bar_mma, phase)) {
      atomicCAS(err, 0, 2);
      ok = false;
    }
    phase ^= 1u;
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
  }
  tc_fence_after();
  // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), 16 columns per load
  const int row = mt * TM + warp * 32 + lane;
  if (ok) {
    for (int cb = 0; cb < TN; cb += 16) {
      float v[16];
      tmem_ld16(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      if (row >= Mdim) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int c = c0 + cb + i;
        if (c >= ncol) break;
        if (MODE == 0) {
          G[((size_t)row * L2 + l * l) * sh.S + c] = v[i];
        } else {
          const int mi = c / sh.S, s = c - mi * sh.S;
          const size_t a = (size_t)(l * l + mi) * sh.N + row;
          const size_t o = a + (size_t)s * ep.ld_out;
          float z = v[i];
          if (ep.mode == EP_PLAIN) {
            ep.out[o] = z;
            continue;
          }
          const float x = ep.X[a + (size_t)s * ep.ld];
          float hx = ep.half_lambda[a] * x + z;
          if (ep.kb) hx += ep.kb[a + (size_t)s * ep.kb_ld];
          if (ep.mode == EP_APPLY) {
            ep.out[o] = hx;
          } else {
            float y = ep.cA * (hx - ep.cshift * x);
            if (ep.Yprev) y -= ep.cB * ep.Yprev[o];
            ep.out[o] = y;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_d, TN);
}

}  // namespace

// ------------------------------------------------------------------ host side
// Split-BF16 tables in the canonical layout: [l][m_tile][k chunk][hi|lo][TM x KC].
// synthesis: rows k (M = n_r), K = n ; analysis: rows n (M = N), K = k.
void build_tc_tables(const HostTables& H, int mode, std::vector<uint16_t>& out, int& m_tiles,
                     int& kpad) {
  const int M = (mode == 0) ? H.n_r : H.N;
  const int K = (mode == 0) ? H.N : H.n_r;
  m_tiles = (M + TM - 1) / TM;
  kpad = ((K + KC - 1) / KC) * KC;
  const int nchunks = kpad / KC;
  const size_t per_chunk = (size_t)2 * TM * KC;
  out.assign((size_t)H.L * m_tiles * nchunks * per_chunk, 0);
  auto bf16_bits = [](float f) -> uint16_t {
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t*>(&b);
  };
  for (int l = 0; l < H.L; ++l)
    for (int mt = 0; mt < m_tiles; ++mt)
      for (int ch = 0; ch < nchunks; ++ch) {
        uint16_t* base = out.data() + ((size_t)(l * m_tiles + mt) * nchunks + ch) * per_chunk;
        for (int r = 0; r < TM; ++r)
          for (int kk = 0; kk < KC; ++kk) {
            const int row = mt * TM + r, k = ch * KC + kk;
            float v = 0.f;
            if (row < M && k < K) {
              const int kr = (mode == 0) ? row : k;  // radial node
              const int n = (mode == 0) ? k : row;   // radial function
              v = (float)H.rad[((size_t)l * H.n_r + kr) * H.N + n];
            }
            const __nv_bfloat16 hb = __float2bfloat16_rn(v);
            const float lo = v - __bfloat162float(hb);
            const int off = canon_off(r, kk, TM) / 2;
            base[off] = bf16_bits(v);
            base[TM * KC + off] = bf16_bits(lo);
          }
      }
}

static int tc_col_tiles(int L, int S) {
  int t = 0;
  for (int l = 0; l < L; ++l) t += ((2 * l + 1) * S + TN - 1) / TN;
  return t;
}

constexpr int kSmemBytes = 4 * TM * KC * 2;

cudaError_t launch_tc_radial_synth(const TcTables& tt, const HostTables& H, const float* X,
                                   long long ldx, float* G, int S, int* err,
                                   cudaStream_t stream) {
  TcShape sh{H.L, H.N, H.n_r, S, tt.m_tiles_synth, tt.kpad_synth};
  dim3 grid(tc_col_tiles(H.L, S), sh.m_tiles);
  Epilogue<float> ep;
  const __nv_bfloat16* tab = static_cast<const __nv_bfloat16*>(tt.synth);
  cudaError_t e = cudaFuncSetAttribute(k_tc_radial<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  k_tc_radial<0><<<grid, kThreads, kSmemBytes, stream>>>(sh, tab, X, ldx, G, ep, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_radial_anal(const TcTables& tt, const HostTables& H, const float* G, int S,
                                  const Epilogue<float>& ep, int* err, cudaStream_t stream) {
  TcShape sh{H.L, H.N, H.n_r, S, tt.m_tiles_anal, tt.kpad_anal};
  dim3 grid(tc_col_tiles(H.L, S), sh.m_tiles);
  const __nv_bfloat16* tab = static_cast<const __nv_bfloat16*>(tt.anal);
  cudaError_t e = cudaFuncSetAttribute(k_tc_radial<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  k_tc_radial<1><<<grid, kThreads, kSmemBytes, stream>>>(sh, tab, nullptr, 0,
                                                          const_cast<float*>(G), ep, err);
  return cudaGetLastError();
}

}  // namespace cs
