// Per-l radial contractions of H.X (Sec. 2.2.2 eqs. G_lmr and Arlm_to_coeff) on the 5th-
// generation tensor cores (tcgen05, sm_103a), for the mixed-precision filter. Each CTA computes
// a tile of 128 state columns c = (m, s) of one l:
//   synthesis : D[c][k] = sum_n X[alpha(l,m,n), s] R_ln(r_k)     -> G[k][l^2 + m][s]
//   analysis  : D[c][n] = sum_k G'[k][l^2 + m][s] R_ln(r_k)      -> Z[alpha(l,m,n), s] (epilogue)
// The state tile is the MMA's A operand (M = 128 columns, K = n or k), the radial table its B
// operand (N = n_r or N rounded up to 16, at most 256), so no tile rows are wasted on the short
// radial dimensions and, in the epilogue, a lane owns one column: the synthesis stores of G
// coalesce across lanes, and the analysis reads and writes 16-byte runs of its column.
// Operands are BF16 in the canonical K-major no-swizzle layout (8-row x 16-byte core
// matrices). Each FP32 operand is split into hi = bf16(x) and lo = bf16(x - hi); the product
// is accumulated in FP32 tensor memory as hi*hi + hi*lo + lo*hi (split BF16), so the
// contraction keeps about 16 significant bits instead of 8.
// The radial tables are pre-split and pre-laid-out at set-up and copied to shared memory with
// cp.async.bulk (TMA engine) per K chunk; the state tile is converted while it is staged. One
// thread issues tcgen05.mma; completion is signalled through an mbarrier (tcgen05.commit);
// four warps read the accumulator back with tcgen05.ld (warp w owns TMEM lanes 32w .. 32w+31 =
// the tile's columns) and run the epilogue of hx_kernels.cuh.
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

constexpr int TC = 128;   // MMA M: state columns per tile
constexpr int KC = 64;    // K elements per shared-memory chunk (4 MMA K-steps of 16)
constexpr int kThreads = 128;
constexpr int kMaxRows = 256;  // MMA N limit (radial rows of the table)

using namespace tcx;

struct TcShape {
  int L, N, n_r, S;
  int rows;      // table rows = output radial dimension rounded up to 16 (MMA N)
  int kpad;      // K rounded up to KC
};

__device__ __forceinline__ void locate_tile(int tile, int S, int& l, int& c0) {
  l = 0;
  for (;;) {
    int ct = ((2 * l + 1) * S + TC - 1) / TC;
    if (tile < ct) break;
    tile -= ct;
    ++l;
  }
  c0 = tile * TC;
}

__host__ __device__ inline uint32_t tmem_cols_for(int rows) {
  uint32_t c = 32;
  while ((int)c < rows) c <<= 1;
  return c;
}

// MODE 0: synthesis (A from X, output G); MODE 1: analysis (A from G, epilogue to X layout)
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_tc_radial(TcShape sh,
                                                         const __nv_bfloat16* __restrict__ tab,
                                                         const float* __restrict__ X,
                                                         long long ldx, float* __restrict__ G,
                                                         Epilogue<float> ep,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];  // A hi, lo: TC x KC; B hi, lo: rows x KC
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t tmem_base_sh;
  const int rows = sh.rows;
  __nv_bfloat16* Bhi = reinterpret_cast<__nv_bfloat16*>(smem);   // table chunk (bulk copy)
  __nv_bfloat16* Blo = Bhi + (size_t)rows * KC;
  __nv_bfloat16* Ahi = Blo + (size_t)rows * KC;                  // state tile
  __nv_bfloat16* Alo = Ahi + TC * KC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int l, c0;
  locate_tile(blockIdx.x, sh.S, l, c0);
  const int ncol = (2 * l + 1) * sh.S;
  const int L2 = sh.L * sh.L;
  const int Kdim = (MODE == 0) ? sh.N : sh.n_r;     // true K
  const int Mout = (MODE == 0) ? sh.n_r : sh.N;     // true output radial dimension
  // 16-byte vector access to X rows (synthesis staging) needs 16-byte aligned rows
  const bool vec_ok = MODE == 0 && (sh.N % 4) == 0 && (ldx % 4) == 0 &&
                      ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  // 16-byte runs in the analysis epilogue: rows of N and all leading dimensions multiples of 4
  const bool vec_ep = MODE == 1 && (sh.N % 4) == 0 && (ep.ld % 4) == 0 && (ep.ld_out % 4) == 0 &&
                      (!ep.kb || (ep.kb_ld % 4) == 0) && (!ep.src || (ep.src_ld % 4) == 0) &&
                      ((reinterpret_cast<uintptr_t>(ep.out) | reinterpret_cast<uintptr_t>(ep.X) |
                        reinterpret_cast<uintptr_t>(ep.half_lambda) |
                        reinterpret_cast<uintptr_t>(ep.kb) | reinterpret_cast<uintptr_t>(ep.src) |
                        reinterpret_cast<uintptr_t>(ep.Yprev)) & 15) == 0;
  const uint32_t bar_tma = smem_u32(&bars[0]);
  const uint32_t bar_mma = smem_u32(&bars[1]);
  const uint32_t tcols = tmem_cols_for(rows);
  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base_sh), tcols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = tmem_base_sh;
  const uint32_t idesc = make_idesc(TC, rows);
  bool ok = true;
  uint32_t phase = 0;
  // table layout: [l][k chunk][hi|lo][rows x KC canonical]
  const int nchunks = sh.kpad / KC;
  const size_t chunk_elems = (size_t)2 * rows * KC;
  const __nv_bfloat16* tab_l = tab + (size_t)l * nchunks * chunk_elems;

  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int kb = ch * KC;
    if (tid == 0) {
      mbar_expect_tx(bar_tma, (uint32_t)(chunk_elems * 2));
      bulk_g2s(smem_u32(Bhi), tab_l + (size_t)ch * chunk_elems, (uint32_t)(chunk_elems * 2),
               bar_tma);
    }
    // stage A (TC rows = state columns, KC K-elements) as split BF16
    // every load of the chunk is issued before any value is converted, so that a thread
    // has all of them in flight at once (the epilogue's stores may alias the inputs, which
    // keeps the compiler from reordering loads past stores by itself)
    constexpr int NT = TC * (KC / 8) / kThreads;  // tasks (8 values each) per thread
    static_assert(NT == 8, "one column (analysis) or one octet of 8 columns (synthesis)");
    float v[NT][8];
    if (MODE == 0) {
      // A[c][n] = X[(l^2 + mi) N + n + s ldx]; task = (column cc, octet oc of n). In one store
      // instruction lanes 8q .. 8q+7 take eight consecutive columns of one octet, whose 16-byte
      // runs are adjacent in the canonical layout (no bank conflicts); four lanes cover 128
      // contiguous bytes of each column in the loads.
      const int warp_id = tid >> 5, ln = tid & 31;
#pragma unroll
      for (int u = 0; u < NT; ++u) {
        const int cc = (warp_id * 4 + (u >> 1)) * 8 + (ln & 7);
        const int oc = (u & 1) * 4 + (ln >> 3), n0 = kb + oc * 8;
        const int c = c0 + cc;
#pragma unroll
        for (int i = 0; i < 8; ++i) v[u][i] = 0.f;
        if (c < ncol) {
          const int mi = c / sh.S, s = c - mi * sh.S;
          const float* src = X + (size_t)(l * l + mi) * sh.N + (size_t)s * ldx + n0;
          if (vec_ok && n0 + 8 <= Kdim) {  // two 16-byte loads (aligned: N, ldx, n0 multiples of 4)
            const float4 a = *reinterpret_cast<const float4*>(src);
            const float4 b = *reinterpret_cast<const float4*>(src + 4);
            v[u][0] = a.x; v[u][1] = a.y; v[u][2] = a.z; v[u][3] = a.w;
            v[u][4] = b.x; v[u][5] = b.y; v[u][6] = b.z; v[u][7] = b.w;
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (n0 + i < Kdim) v[u][i] = src[i];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < NT; ++u) {
        const int cc = (warp_id * 4 + (u >> 1)) * 8 + (ln & 7);
        const int oc = (u & 1) * 4 + (ln >> 3);
        __align__(16) __nv_bfloat16 h[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split_bf16(v[u][i], h[i], lo[i]);
        const int off = canon_off(cc, oc * 8, TC);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Ahi) + off) =
            *reinterpret_cast<uint4*>(h);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Alo) + off) =
            *reinterpret_cast<uint4*>(lo);
      }
    } else {
      // A[c][k] = G[(k L^2 + l^2) S + c]; thread = column cc = tid, all eight k octets
      const int cc = tid, c = c0 + cc;
#pragma unroll
      for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = kb + u * 8 + i;
          v[u][i] = (c < ncol && k < Kdim) ? G[((size_t)k * L2 + l * l) * sh.S + c] : 0.f;
        }
#pragma unroll
      for (int u = 0; u < NT; ++u) {
        __align__(16) __nv_bfloat16 h[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split_bf16(v[u][i], h[i], lo[i]);
        const int off = canon_off(cc, u * 8, TC);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Ahi) + off) =
            *reinterpret_cast<uint4*>(h);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Alo) + off) =
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
          const uint32_t ao = ks * (TC / 8) * 256, bo = ks * (rows / 8) * 256;
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
  // epilogue: warp w reads TMEM lanes 32w..32w+31 (the tile's columns), 16 radial rows per
  // load; thread = one column c
  const int c = c0 + warp * 32 + lane;
  const bool live = ok && c < ncol;
  int mi = 0, s = 0;
  if (c < ncol) {
    mi = c / sh.S;
    s = c - mi * sh.S;
  }
  // weight of the residual-form source term of this column (0 when there is none)
  const float sw = (MODE == 1 && ep.src && c < ncol) ? ep.src_w[s] : 0.f;
  if (ok) {
    for (int rb = 0; rb < rows; rb += 16) {
      float v[16];
      tmem_ld16(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)rb, v);
      if (!live) continue;
      if (MODE == 0) {
        // G[k][l^2 + mi][s] for k = rb .. rb + 15: lanes (consecutive c) write consecutive words
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int k = rb + i;
          if (k < Mout) G[((size_t)k * L2 + l * l) * sh.S + c] = v[i];
        }
        continue;
      }
      // Z[alpha(l, mi, n), s] for n = rb .. rb + 15 (contiguous in n)
      const size_t a0 = (size_t)(l * l + mi) * sh.N;
      if (vec_ep && rb + 16 <= Mout) {
        // 16-byte runs: four float4 of each operand (a0 + rb, s ld, s ld_out multiples of 4)
        const size_t a = a0 + rb;
        const size_t o = a + (size_t)s * ep.ld_out;
        float4* out4 = reinterpret_cast<float4*>(ep.out + o);
        if (ep.mode == EP_PLAIN) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            out4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          continue;
        }
        const float4* x4 = reinterpret_cast<const float4*>(ep.X + a + (size_t)s * ep.ld);
        const float4* h4 = reinterpret_cast<const float4*>(ep.half_lambda + a);
        const float4* k4 =
            ep.kb ? reinterpret_cast<const float4*>(ep.kb + a + (size_t)s * ep.kb_ld) : nullptr;
        const float4* y4 =
            ep.Yprev ? reinterpret_cast<const float4*>(ep.Yprev + o) : nullptr;
        const float4* s4 =
            ep.src ? reinterpret_cast<const float4*>(ep.src + a + (size_t)s * ep.src_ld) : nullptr;
        // all loads of the run first (out may alias Yprev: no store before the last load)
        float4 xv[4], hv[4], kv[4], yv[4], sv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xv[q] = x4[q];
          hv[q] = h4[q];
          kv[q] = k4 ? k4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
          yv[q] = (y4 && ep.mode != EP_APPLY) ? y4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
          sv[q] = s4 ? s4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float xs[4] = {xv[q].x, xv[q].y, xv[q].z, xv[q].w};
          const float hs[4] = {hv[q].x, hv[q].y, hv[q].z, hv[q].w};
          const float ks[4] = {kv[q].x, kv[q].y, kv[q].z, kv[q].w};
          const float ys[4] = {yv[q].x, yv[q].y, yv[q].z, yv[q].w};
          const float ss[4] = {sv[q].x, sv[q].y, sv[q].z, sv[q].w};
          float r[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float hx = fmaf(hs[j], xs[j], v[4 * q + j]);
            if (k4) hx = __fadd_rn(hx, ks[j]);
            if (s4) hx = fmaf(sw, ss[j], hx);
            if (ep.mode == EP_APPLY) {
              r[j] = hx;
            } else {
              float y = __fmul_rn(ep.cA, fmaf(-ep.cshift, xs[j], hx));
              if (y4) y = fmaf(-ep.cB, ys[j], y);
              r[j] = y;
            }
          }
          out4[q] = make_float4(r[0], r[1], r[2], r[3]);
        }
        continue;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = rb + i;
        if (n >= Mout) break;
        const size_t a = a0 + n;
        const size_t o = a + (size_t)s * ep.ld_out;
        const float z = v[i];
        if (ep.mode == EP_PLAIN) {
          ep.out[o] = z;
          continue;
        }
        // the same roundings as the FP32 radial tiles (fmaf, __fmul_rn, __fadd_rn)
        const float x = ep.X[a + (size_t)s * ep.ld];
        float hx = fmaf(ep.half_lambda[a], x, z);
        if (ep.kb) hx = __fadd_rn(hx, ep.kb[a + (size_t)s * ep.kb_ld]);
        if (ep.src) hx = fmaf(sw, ep.src[a + (size_t)s * ep.src_ld], hx);
        if (ep.mode == EP_APPLY) {
          ep.out[o] = hx;
        } else {
          float y = __fmul_rn(ep.cA, fmaf(-ep.cshift, x, hx));
          if (ep.Yprev) y = fmaf(-ep.cB, ep.Yprev[o], y);
          ep.out[o] = y;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_d, tcols);
}

}  // namespace

// ------------------------------------------------------------------ host side
// Split-BF16 tables in the canonical layout: [l][k chunk][hi|lo][rows x KC], rows = the output
// radial dimension rounded up to 16 (synthesis: k < n_r, K = n; analysis: n < N, K = k).
void build_tc_tables(const HostTables& H, int mode, std::vector<uint16_t>& out, int& rows,
                     int& kpad) {
  const int M = (mode == 0) ? H.n_r : H.N;
  const int K = (mode == 0) ? H.N : H.n_r;
  rows = ((M + 15) / 16) * 16;
  kpad = ((K + KC - 1) / KC) * KC;
  const int nchunks = kpad / KC;
  const size_t per_chunk = (size_t)2 * rows * KC;
  out.assign((size_t)H.L * nchunks * per_chunk, 0);
  auto bf16_bits = [](float f) -> uint16_t {
    __nv_bfloat16 b = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t*>(&b);
  };
  for (int l = 0; l < H.L; ++l)
    for (int ch = 0; ch < nchunks; ++ch) {
      uint16_t* base = out.data() + ((size_t)l * nchunks + ch) * per_chunk;
      for (int r = 0; r < rows; ++r)
        for (int kk = 0; kk < KC; ++kk) {
          const int k = ch * KC + kk;
          float v = 0.f;
          if (r < M && k < K) {
            const int kr = (mode == 0) ? r : k;  // radial node
            const int n = (mode == 0) ? k : r;   // radial function
            v = (float)H.rad[((size_t)l * H.n_r + kr) * H.N + n];
          }
          const __nv_bfloat16 hb = __float2bfloat16_rn(v);
          const float lo = v - __bfloat162float(hb);
          const int off = canon_off(r, kk, rows) / 2;
          base[off] = bf16_bits(v);
          base[(size_t)rows * KC + off] = bf16_bits(lo);
        }
    }
}

static int tc_col_tiles(int L, int S) {
  int t = 0;
  for (int l = 0; l < L; ++l) t += ((2 * l + 1) * S + TC - 1) / TC;
  return t;
}

static size_t smem_bytes(int rows) { return (size_t)2 * (rows + TC) * KC * 2; }

bool tc_radial_fits(const HostTables& H) {
  return ((H.n_r + 15) / 16) * 16 <= kMaxRows && ((H.N + 15) / 16) * 16 <= kMaxRows;
}

cudaError_t launch_tc_radial_synth(const TcTables& tt, const HostTables& H, const float* X,
                                   long long ldx, float* G, int S, int* err,
                                   cudaStream_t stream) {
  if (tt.rows_synth > kMaxRows) return cudaErrorInvalidConfiguration;
  TcShape sh{H.L, H.N, H.n_r, S, tt.rows_synth, tt.kpad_synth};
  dim3 grid(tc_col_tiles(H.L, S));
  Epilogue<float> ep;
  const __nv_bfloat16* tab = static_cast<const __nv_bfloat16*>(tt.synth);
  const size_t smem = smem_bytes(sh.rows);
  cudaError_t e = cudaFuncSetAttribute(k_tc_radial<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_radial<0><<<grid, kThreads, smem, stream>>>(sh, tab, X, ldx, G, ep, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_radial_anal(const TcTables& tt, const HostTables& H, const float* G, int S,
                                  const Epilogue<float>& ep, int* err, cudaStream_t stream) {
  if (tt.rows_anal > kMaxRows) return cudaErrorInvalidConfiguration;
  TcShape sh{H.L, H.N, H.n_r, S, tt.rows_anal, tt.kpad_anal};
  dim3 grid(tc_col_tiles(H.L, S));
  const __nv_bfloat16* tab = static_cast<const __nv_bfloat16*>(tt.anal);
  const size_t smem = smem_bytes(sh.rows);
  cudaError_t e = cudaFuncSetAttribute(k_tc_radial<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_tc_radial<1><<<grid, kThreads, smem, stream>>>(sh, tab, nullptr, 0,
                                                          const_cast<float*>(G), ep, err);
  return cudaGetLastError();
}

}  // namespace cs
