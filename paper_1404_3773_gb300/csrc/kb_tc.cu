// Kleinman-Bylander projector pair of H.X (Sec. 2.3.2: the non-local term is a pair of
// matrix products with the projector coefficients) on the tcgen05 tensor cores, for the
// mixed-precision filter:
//   W = P^T X              (n_p x S;  K = d, split over K across CTAs, partials summed in a
//                           fixed order, then scaled by the couplings h)
//   Z = P (h W)            (d x S;    K = n_p)
// Both products are split-BF16 (each FP32 operand = hi + lo, accumulated in FP32 tensor
// memory as hi*hi + hi*lo + lo*hi). The projector tables are split and laid out once, when
// the projectors are set; the state block is split by one conversion kernel per call.
// Operand tiles are stored chunk by chunk ([tile of 128 rows][K chunk of 64][hi|lo][128 x 64
// canonical]) so that every pipeline stage is two contiguous 32 KB bulk copies. Each CTA runs
// a three-stage pipeline: one thread issues the bulk copies (cp.async.bulk, completion on
// an mbarrier), one thread issues the MMAs and releases stages through tcgen05.commit, and
// four warps read the accumulator back. Every wait is bounded; on expiry the kernel records
// an error code, waits (bounded) for its copies still in flight, frees its tensor memory and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kb_tc.h"
#include "tc_common.cuh"

namespace cs {

namespace {

using namespace tcx;

constexpr int TM = 128, TN = 128, KC = 64, STAGES = 3, kThreads = 128;
constexpr int kHalf = TM * KC * 2;        // bytes of hi (or lo) of one operand chunk
constexpr int kOpChunk = 2 * kHalf;       // hi + lo = 32 KB
constexpr int kSmem = STAGES * 2 * kOpChunk;  // A and B per stage = 192 KB
constexpr int kSms = 152;

enum { EPI_PARTIAL = 0, EPI_STORE = 1 };

struct GemmArgs {
  const unsigned char* A;  // [m tile][kchunks][hi|lo][TM x KC]
  const unsigned char* B;  // [n tile][kchunks][hi|lo][TN x KC]
  int kchunks, kper;       // chunks per operand tile; chunks per CTA along grid.z
  long long M;             // true rows (EPI_STORE guard)
  int N;                   // true columns (EPI_STORE guard)
  float* out;
  long long ld_out;        // EPI_STORE: out[row + col ld_out]; EPI_PARTIAL: row stride
  long long z_stride;      // EPI_PARTIAL: stride between K splits
  int* err;
};

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm(GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int consumed_sh, flag_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, nt = blockIdx.y, z = blockIdx.z;
  const int k0 = z * g.kper;
  const int k1 = min(g.kchunks, k0 + g.kper);
  const int nk = max(0, k1 - k0);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    consumed_sh = 0;
    flag_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base_sh), TN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_d = tmem_base_sh;
  const unsigned char* Ab = g.A + (size_t)mt * g.kchunks * kOpChunk;
  const unsigned char* Bb = g.B + (size_t)nt * g.kchunks * kOpChunk;
  auto sA = [&](int s) { return smem_u32(smem + (size_t)s * 2 * kOpChunk); };
  auto sB = [&](int s) { return smem_u32(smem + (size_t)s * 2 * kOpChunk + kOpChunk); };
  int issued = 0;
  if (tid == 0) {
    // producer: stage s is refilled once the MMAs that read it have completed
    for (int i = 0; i < nk; ++i) {
      const int s = i % STAGES;
      if (i >= STAGES && !mbar_wait(smem_u32(&empty[s]), ((i / STAGES) - 1) & 1)) {
        atomicCAS(g.err, 0, 3);
        flag_sh = 1;
        break;
      }
      mbar_expect_tx(smem_u32(&full[s]), 2 * kOpChunk);
      bulk_g2s(sA(s), Ab + (size_t)(k0 + i) * kOpChunk, kOpChunk, smem_u32(&full[s]));
      bulk_g2s(sB(s), Bb + (size_t)(k0 + i) * kOpChunk, kOpChunk, smem_u32(&full[s]));
      issued = i + 1;
    }
  } else if (tid == 32) {
    // MMA issuer
    constexpr uint32_t idesc = make_idesc(TM, TN);
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % STAGES;
      if (!mbar_wait(smem_u32(&full[s]), (i / STAGES) & 1)) {
        atomicCAS(g.err, 0, 4);
        flag_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t a_hi = sA(s), a_lo = a_hi + kHalf, b_hi = sB(s), b_lo = b_hi + kHalf;
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
        const uint32_t ao = ks * (TM / 8) * 256, bo = ks * (TN / 8) * 256;
        const uint64_t dah = make_desc(a_hi + ao, 128, 256), dal = make_desc(a_lo + ao, 128, 256);
        const uint64_t dbh = make_desc(b_hi + bo, 128, 256), dbl = make_desc(b_lo + bo, 128, 256);
        mma_bf16(tmem_d, dah, dbh, idesc, (i > 0 || ks > 0) ? 1u : 0u);
        mma_bf16(tmem_d, dah, dbl, idesc, 1u);
        mma_bf16(tmem_d, dal, dbh, idesc, 1u);
      }
      mma_commit(smem_u32(&empty[s]));
    }
    consumed_sh = i;
    mma_commit(smem_u32(&done));  // arrives when every MMA issued above has completed
  }
  __syncwarp();
  bool ok = mbar_wait(smem_u32(&done), 0);
  if (!ok) atomicCAS(g.err, 0, 5);
  __syncthreads();
  if (tid == 0 && flag_sh) {
    // error path: let the copies that no MMA consumed land before the CTA exits
    for (int i = consumed_sh; i < issued; ++i)
      mbar_wait(smem_u32(&full[i % STAGES]), (i / STAGES) & 1);
  }
  ok = ok && !flag_sh;
  tc_fence_after();
  const long long row = (long long)mt * TM + warp * 32 + lane;
  for (int cb = 0; cb < TN; cb += 16) {
    float v[16];
    if (ok && nk > 0) {
      tmem_ld16(tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = 0.f;
    }
    const int c0 = nt * TN + cb;
    if (EPI == EPI_PARTIAL) {
      float4* p = reinterpret_cast<float4*>(g.out + (size_t)z * g.z_stride + row * g.ld_out + c0);
#pragma unroll
      for (int i = 0; i < 4; ++i) p[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    } else if (row < g.M) {
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (c0 + i < g.N) g.out[row + (size_t)(c0 + i) * g.ld_out] = v[i];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem_d, TN);
}

__device__ __forceinline__ void store_split8(unsigned char* chunk, int row, int k8,
                                             const float* v) {
  __align__(16) __nv_bfloat16 h[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) split_bf16(v[i], h[i], lo[i]);
  const int off = canon_off(row, k8, TM);
  *reinterpret_cast<uint4*>(chunk + off) = *reinterpret_cast<const uint4*>(h);
  *reinterpret_cast<uint4*>(chunk + kHalf + off) = *reinterpret_cast<const uint4*>(lo);
}

// Operand rows = columns j of a column-major matrix src (element (i, j) = src[i + j ld]),
// K = i. One thread per (operand row, octet of K); consecutive threads take consecutive rows.
template <typename Tin>
__global__ void k_split_cols(const Tin* __restrict__ src, long long ld, long long nK, int nrows,
                             int rtiles, int kchunks, unsigned char* __restrict__ op) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long rows_pad = (long long)rtiles * TM;
  if (t >= rows_pad * kchunks * (KC / 8)) return;
  const int r = (int)(t % rows_pad);
  const long long oct = t / rows_pad;
  const long long k0 = oct * 8;
  float v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long k = k0 + i;
    v[i] = (r < nrows && k < nK) ? (float)src[k + (long long)r * ld] : 0.f;
  }
  const int tile = r / TM;
  const long long ch = k0 / KC;
  unsigned char* chunk = op + ((size_t)tile * kchunks + ch) * kOpChunk;
  store_split8(chunk, r % TM, (int)(k0 % KC), v);
}

// Operand rows = rows i of a column-major matrix src, K = columns j.
template <typename Tin>
__global__ void k_split_rows(const Tin* __restrict__ src, long long ld, long long nrows, int nK,
                             long long rtiles, int kchunks, unsigned char* __restrict__ op) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long rows_pad = rtiles * TM;
  if (t >= rows_pad * kchunks * (KC / 8)) return;
  const long long r = t % rows_pad;
  const int oct = (int)(t / rows_pad);
  const int k0 = oct * 8;
  float v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = k0 + i;
    v[i] = (r < nrows && k < nK) ? (float)src[r + (long long)k * ld] : 0.f;
  }
  const long long tile = r / TM;
  unsigned char* chunk = op + ((size_t)tile * kchunks + k0 / KC) * kOpChunk;
  store_split8(chunk, (int)(r % TM), k0 % KC, v);
}

// W[p][s] = h[p] * sum_z partial[z][p][s] (fixed order over z), written as the B operand of
// the second product: operand rows = s, K = p. One thread per (s, octet of p).
__global__ void k_kb_reduce(const float* __restrict__ partial, int ksplit, long long z_stride,
                            int ldp, const float* __restrict__ h, int n_p, int S, int stiles,
                            int kchunks, unsigned char* __restrict__ op) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int rows_pad = stiles * TN;
  if (t >= rows_pad * kchunks * (KC / 8)) return;
  const int s = t % rows_pad;
  const int p0 = (t / rows_pad) * 8;
  float v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int p = p0 + i;
    float acc = 0.f;
    if (s < S && p < n_p) {
      for (int zz = 0; zz < ksplit; ++zz) acc += partial[(size_t)zz * z_stride + (size_t)p * ldp + s];
      acc *= h[p];
    }
    v[i] = acc;
  }
  unsigned char* chunk = op + ((size_t)(s / TN) * kchunks + p0 / KC) * kOpChunk;
  store_split8(chunk, s % TN, p0 % KC, v);
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

KbTcShape kb_tc_shape(long long d, int n_p, int S) {
  KbTcShape s;
  s.d = d;
  s.n_p = n_p;
  s.S = S;
  s.mtA = (n_p + TM - 1) / TM;
  s.kchA = (int)((d + KC - 1) / KC);
  s.mtB = (d + TM - 1) / TM;
  s.kchB = (n_p + KC - 1) / KC;
  s.stiles = (S + TN - 1) / TN;
  int tiles = s.mtA * s.stiles;
  s.ksplit = tiles >= kSms ? 1 : kSms / tiles;
  if (s.ksplit > s.kchA) s.ksplit = s.kchA;
  s.kper = (s.kchA + s.ksplit - 1) / s.ksplit;
  s.ksplit = (s.kchA + s.kper - 1) / s.kper;
  s.tabA_bytes = (size_t)s.mtA * s.kchA * kOpChunk;
  s.tabB_bytes = (size_t)s.mtB * s.kchB * kOpChunk;
  s.xc_bytes = (size_t)s.stiles * s.kchA * kOpChunk;
  s.wc_bytes = (size_t)s.stiles * s.kchB * kOpChunk;
  s.part_bytes = (size_t)s.ksplit * s.mtA * TM * s.stiles * TN * sizeof(float);
  return s;
}

size_t kb_tc_work_bytes(const KbTcShape& s) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  return al(s.xc_bytes) + al(s.wc_bytes) + al(s.part_bytes);
}

cudaError_t build_kb_tc_tables(const double* pcoef, long long d, int n_p, void* tabA, void* tabB,
                               cudaStream_t stream) {
  const KbTcShape s = kb_tc_shape(d, n_p, 1);
  // first product: operand rows = projectors (columns of P), K = basis index
  long long nA = (long long)s.mtA * TM * s.kchA * (KC / 8);
  k_split_cols<double><<<blocks_for(nA, 256), 256, 0, stream>>>(
      pcoef, d, d, n_p, s.mtA, s.kchA, static_cast<unsigned char*>(tabA));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // second product: operand rows = basis index (rows of P), K = projectors
  long long nB = s.mtB * TM * s.kchB * (KC / 8);
  k_split_rows<double><<<blocks_for(nB, 256), 256, 0, stream>>>(
      pcoef, d, d, n_p, s.mtB, s.kchB, static_cast<unsigned char*>(tabB));
  return cudaGetLastError();
}

cudaError_t launch_kb_tc(const void* tabA, const void* tabB, const KbTcShape& s, const float* X,
                         long long ldx, const float* h, float* Z, long long ldz, void* work,
                         int* err, cudaStream_t stream, int* launches) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  unsigned char* xc = static_cast<unsigned char*>(work);
  unsigned char* wc = xc + al(s.xc_bytes);
  float* part = reinterpret_cast<float*>(wc + al(s.wc_bytes));
  cudaError_t e;
  for (auto fn : {(const void*)k_tc_gemm<EPI_PARTIAL>, (const void*)k_tc_gemm<EPI_STORE>}) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
  }
  // 1. split the state block: operand rows = states, K = basis index
  long long nx = (long long)s.stiles * TN * s.kchA * (KC / 8);
  k_split_cols<float><<<blocks_for(nx, 256), 256, 0, stream>>>(X, ldx, s.d, s.S, s.stiles,
                                                               s.kchA, xc);
  // 2. partial W = P^T X over K splits
  GemmArgs g1{};
  g1.A = static_cast<const unsigned char*>(tabA);
  g1.B = xc;
  g1.kchunks = s.kchA;
  g1.kper = s.kper;
  g1.M = (long long)s.mtA * TM;
  g1.N = s.stiles * TN;
  g1.out = part;
  g1.ld_out = (long long)s.stiles * TN;
  g1.z_stride = (long long)s.mtA * TM * s.stiles * TN;
  g1.err = err;
  k_tc_gemm<EPI_PARTIAL><<<dim3(s.mtA, s.stiles, s.ksplit), kThreads, kSmem, stream>>>(g1);
  // 3. W = h * sum of partials, as the split operand of the second product
  long long nw = (long long)s.stiles * TN * s.kchB * (KC / 8);
  k_kb_reduce<<<blocks_for(nw, 256), 256, 0, stream>>>(part, s.ksplit, g1.z_stride,
                                                       (int)g1.ld_out, h, s.n_p, s.S, s.stiles,
                                                       s.kchB, wc);
  // 4. Z = P (h W)
  GemmArgs g2{};
  g2.A = static_cast<const unsigned char*>(tabB);
  g2.B = wc;
  g2.kchunks = s.kchB;
  g2.kper = s.kchB;
  g2.M = s.d;
  g2.N = s.S;
  g2.out = Z;
  g2.ld_out = ldz;
  g2.err = err;
  k_tc_gemm<EPI_STORE><<<dim3((unsigned)s.mtB, s.stiles, 1), kThreads, kSmem, stream>>>(g2);
  if (launches) *launches = 4;
  return cudaGetLastError();
}

}  // namespace cs
