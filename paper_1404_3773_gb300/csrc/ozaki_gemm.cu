// FP64 matrix products of the dense steps (Sec. 3.2.1: the Gram matrices of Cholesky-QR and
// Rayleigh-Ritz and the rotations by their small factors) from exact products of small-integer
// slices on the tcgen05 tensor cores: the error-free splitting of Ozaki, Ogita, Oishi and Rump
// (2012) in its integer-slice form (ozaki_split.cuh).
//
//   C = A^T B (Gram: one exponent per column of A and of B) or C = A Q (rotation: one exponent
//   per row of A, per column of Q). Each FP64 operand value becomes s = 8 integer digits of
//   beta = 7 bits (|digit| <= 64, exact in BF16) below its row's or column's power of two.
//   The product of digit matrices k and l carries the unit 2^(E + F - 12 - 7 (k + l)); the
//   pairs with k + l <= 7 are kept. All pairs on one diagonal t = k + l share that unit, so
//   each diagonal has one FP32 accumulator in tensor memory: a row adds at most 8 products of
//   magnitude <= 2^12 to it, so over a window of 512 rows every partial sum is an integer of
//   magnitude <= 2^24, held exactly in any order of addition. After each window the eight
//   accumulators are read back and added, as integers, into registers; at the end the exact
//   diagonal sums are combined in 128-bit integers and rounded once to FP64. The result is
//   the exactly rounded value of the truncated slice sum: bit for bit what the oracle computes.
//
// Layout of a split operand: [tile of TR operand rows][K step of 16][digit][group of 8 rows of
// the tile][256 B canonical core-matrix pair] (canonical K-major, no swizzle), TR = 128 for the
// A side and 32 for the B side, so one pipeline stage of a tile (two K steps, all digits) is
// one contiguous run: 64 KB (A) and 16 KB (B), two bulk copies per stage.
//
// The product kernel: one CTA per (128 rows of the A side) x (32 rows of the B side) x (a
// group of up to 64 windows of K). Warp 8 issues the bulk copies (two stages of 32 K rows:
// 80 KB), warp 9 issues the MMAs into one of two tensor-memory buffers of 8 diagonals x 32
// columns, and warps 0-7 drain the other buffer (warps w and w + 4 share a lane quarter and
// take diagonals 0-3 and 4-7). The digits of the B tile sit one after another in shared
// memory, so digit k of A times digits 0 .. 7-k of B is one MMA of N = (8 - k) 32 whose
// columns are the accumulators of diagonals k .. 7: 8 MMAs per K step of 16. Every wait is bounded; on expiry the kernel
// records an error code in *err, lets its copies and MMAs land (bounded), frees its tensor
// memory and returns.
//
// Structure taken where the operands have it (results bit for bit unchanged): a Gram matrix of
// one block with itself runs only the tiles that reach its upper triangle and writes each value
// to both places; a rotation by an upper-triangular factor stops each tile's K range at the
// tile's last column; rotations walk the grid B-side tile first, so the CTAs that read one
// A-side tile run together and share it through L2.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "hx_kernels.cuh"
#include "ozaki_split.cuh"
#include "tc_common.cuh"

namespace cs {

namespace {

using namespace tcx;

constexpr int kBeta = 7, kS = 8;
constexpr int kWin = 512;                 // K rows of one exact FP32 window
constexpr int kKC = 32;                   // K rows per pipeline stage (2 K steps)
constexpr int kChunksPerWin = kWin / kKC; // 16
constexpr int kTM = 128, kTN = 32;        // output tile: A-side rows x B-side rows
constexpr int kMaxWinPerCta = 64;         // int32 window sums stay below 2^30
constexpr int kDrainWarps = 8;
constexpr int kThreads = 32 * (kDrainWarps + 2);
constexpr int kAStep = kTM / 8 * 256;     // bytes of one (K step, digit) A tile: 4 KB
constexpr int kBStep = kTN / 8 * 256;     // 1 KB
constexpr int kStageBytes = 2 * kS * (kAStep + kBStep);  // 80 KB
constexpr int kSmem = 2 * kStageBytes;                     // two stages
constexpr int kTmemCols = 512;            // 2 buffers x 8 diagonals x 32 columns
constexpr int kSms = 152;

struct OzArgs {
  const unsigned char* A;  // split A side
  const unsigned char* B;  // split B side
  long long ksteps;        // K steps of 16 in both layouts (K rows / 16, padded)
  long long kchunks;       // K rows / 32 (padded)
  int wins_per_cta;
  // direct: C[i + j ldc] for i < M, j < N;  partial: part[((z 8 + t) Np + j) Mp + i]
  int direct;
  double* C;
  long long ldc, M;
  int N;
  const int* EA;
  const int* EB;
  int* part;
  long long Mp, Np;
  int* err;
  int sym;     // A and B are one block: only tiles that reach the upper triangle, mirrored
  int upper;   // B is upper triangular: a tile's K range ends at its last column
  int n_fast;  // grid x runs over the B-side tiles (the CTAs of one A tile run together)
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) k_oz_mma(OzArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[2], empty[2], acc_full[2], acc_empty[2], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int flag_sh, issued_sh, consumed_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long mt = g.n_fast ? blockIdx.y : blockIdx.x;
  const int nt = g.n_fast ? blockIdx.x : blockIdx.y, z = blockIdx.z;
  // C = A^T A: a tile wholly below the diagonal is the mirror of one above it (the exact sum
  // of C[i][j] and of C[j][i] is one number), written by that tile
  if (g.sym && mt * kTM > (long long)nt * kTN + kTN - 1) return;
  // upper-triangular B: rows past the tile's last column are zero, their digits add nothing
  const long long kc =
      g.upper ? min(g.kchunks, ((long long)nt * kTN + kTN + kKC - 1) / kKC) : g.kchunks;
  const long long c0 = (long long)z * g.wins_per_cta * kChunksPerWin;
  const long long c1 = min(kc, c0 + (long long)g.wins_per_cta * kChunksPerWin);
  const int nk = (int)max(0ll, c1 - c0);
  const int nw = (nk + kChunksPerWin - 1) / kChunksPerWin;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
      mbar_init(smem_u32(&acc_full[s]), 1);
      mbar_init(smem_u32(&acc_empty[s]), 32 * kDrainWarps);
    }
    mbar_init(smem_u32(&done), 1);
    flag_sh = 0;
    issued_sh = 0;
    consumed_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(smem_u32(&tmem_base_sh), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;
  auto sA = [&](int s) { return smem_u32(smem + (size_t)s * kStageBytes); };
  auto sB = [&](int s) { return smem_u32(smem + (size_t)s * kStageBytes + 2 * kS * kAStep); };
  int acc[4][kTN];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < kTN; ++c) acc[a][c] = 0;
  bool ok = true;

  if (warp == kDrainWarps && lane == 0) {
    // producer: stage s is refilled once the MMAs that read it have completed
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i & 1;
      if (i >= 2 && !mbar_wait(smem_u32(&empty[s]), ((i >> 1) - 1) & 1)) {
        atomicCAS(g.err, 0, 21);
        flag_sh = 1;
        break;
      }
      const uint32_t fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, kStageBytes);
      const long long kstep = (c0 + i) * 2;
      const unsigned char* a = g.A + ((mt * g.ksteps + kstep) * kS) * (size_t)kAStep;
      const unsigned char* b = g.B + (((long long)nt * g.ksteps + kstep) * kS) * (size_t)kBStep;
      bulk_g2s(sA(s), a, 2 * kS * kAStep, fb);
      bulk_g2s(sB(s), b, 2 * kS * kBStep, fb);
    }
    issued_sh = i;
  } else if (warp == kDrainWarps + 1 && lane == 0) {
    // MMA issuer: per K step, digit k of A times digits 0 .. 7-k of B (N = (8 - k) 32) into
    // the accumulators of diagonals k .. 7
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i & 1;
      const int w = i / kChunksPerWin, buf = w & 1;
      const bool first = (i % kChunksPerWin) == 0;
      if (first && w >= 2 && !mbar_wait(smem_u32(&acc_empty[buf]), ((w >> 1) - 1) & 1)) {
        atomicCAS(g.err, 0, 22);
        flag_sh = 1;
        break;
      }
      if (!mbar_wait(smem_u32(&full[s]), (i >> 1) & 1)) {
        atomicCAS(g.err, 0, 23);
        flag_sh = 1;
        break;
      }
      tc_fence_after();
      const uint32_t dbase = tmem + (uint32_t)(buf * kS * kTN);
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t bd = make_desc(sB(s) + ks * kS * kBStep, 128, 256);
#pragma unroll
        for (int k = 0; k < kS; ++k) {
          const uint64_t ad = make_desc(sA(s) + (ks * kS + k) * kAStep, 128, 256);
          const uint32_t idesc = make_idesc(kTM, (kS - k) * kTN);
          // k = 0 covers every diagonal: it starts each window's accumulators
          const uint32_t accum = (!first || ks > 0 || k > 0) ? 1u : 0u;
          mma_bf16(dbase + (uint32_t)(k * kTN), ad, bd, idesc, accum);
        }
      }
      mma_commit(smem_u32(&empty[s]));
      if ((i % kChunksPerWin) == kChunksPerWin - 1 || i == nk - 1)
        mma_commit(smem_u32(&acc_full[buf]));
    }
    consumed_sh = i;
    mma_commit(smem_u32(&done));  // arrives when every MMA issued above has completed
  } else if (warp < kDrainWarps) {
    // drain: warp w reads lanes 32 (w % 4) .. + 31 and diagonals 4 (w / 4) .. + 3
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int t0 = (warp >> 2) * 4;
    for (int w = 0; w < nw; ++w) {
      const int buf = w & 1;
      if (!mbar_wait(smem_u32(&acc_full[buf]), (w >> 1) & 1)) {
        atomicCAS(g.err, 0, 24);
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        float v[kTN];
        const uint32_t col = (uint32_t)(buf * kS * kTN + (t0 + tt) * kTN);
        tmem_ld16_issue(tmem + lane_base + col, v);
        tmem_ld16_issue(tmem + lane_base + col + 16, v + 16);
        tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < kTN; ++c) acc[tt][c] += __float2int_rn(v[c]);
      }
      tc_fence_before();
      mbar_arrive(smem_u32(&acc_empty[buf]));
    }
  }
  __syncwarp();
  // everyone: the MMAs issued have completed
  if (!mbar_wait(smem_u32(&done), 0)) {
    atomicCAS(g.err, 0, 25);
    ok = false;
  }
  __syncthreads();
  if (warp == kDrainWarps && lane == 0 && flag_sh) {
    // error path: let the copies that no MMA consumed land before the CTA exits
    for (int i = consumed_sh; i < issued_sh; ++i)
      mbar_wait(smem_u32(&full[i & 1]), (i >> 1) & 1);
  }
  ok = ok && !flag_sh;
  const int drain_ok = __syncthreads_and((warp < kDrainWarps) ? (ok ? 1 : 0) : 1);
  if (drain_ok && warp < kDrainWarps) {
    const long long i = mt * kTM + (warp & 3) * 32 + lane;  // A-side row
    const int t0 = (warp >> 2) * 4;
    if (!g.direct) {
#pragma unroll
      for (int tt = 0; tt < 4; ++tt)
#pragma unroll
        for (int c = 0; c < kTN; ++c) {
          const long long j = (long long)nt * kTN + c;
          g.part[(((long long)z * kS + t0 + tt) * g.Np + j) * g.Mp + i] = acc[tt][c];
        }
    }
  }
  if (g.direct) {
    // every drain warp combines half of its rows' columns: warps 0-3 (diagonals 0-3) take
    // columns 0-15 and hand diagonals 0-3 of columns 16-31 to warps 4-7, which hand back
    // diagonals 4-7 of columns 0-15 (through shared memory; the stages are idle now)
    constexpr int H = kTN / 2;
    int* lo_part = reinterpret_cast<int*>(smem);   // [4][H][kTM]: diagonals 0-3, columns H..
    int* hi_part = lo_part + 4 * H * kTM;          // [4][H][kTM]: diagonals 4-7, columns 0..
    const int r = (warp & 3) * 32 + lane;
    if (drain_ok && warp < kDrainWarps) {
      if (warp < 4) {
#pragma unroll
        for (int tt = 0; tt < 4; ++tt)
#pragma unroll
          for (int c = 0; c < H; ++c) lo_part[(tt * H + c) * kTM + r] = acc[tt][H + c];
      } else {
#pragma unroll
        for (int tt = 0; tt < 4; ++tt)
#pragma unroll
          for (int c = 0; c < H; ++c) hi_part[(tt * H + c) * kTM + r] = acc[tt][c];
      }
    }
    __syncthreads();
    const long long i = mt * kTM + r;
    if (drain_ok && warp < kDrainWarps && i < g.M) {
      const int ea = g.EA[i];
      const bool low = warp < 4;
      // fully unrolled, so that acc stays in registers
#pragma unroll
      for (int c = 0; c < H; ++c) {
        const long long j = (long long)nt * kTN + (low ? c : H + c);
        if (j < g.N && (!g.sym || i <= j)) {
          int64_t D[kS];
#pragma unroll
          for (int tt = 0; tt < 4; ++tt) {
            D[tt] = low ? acc[tt][c] : lo_part[(tt * H + c) * kTM + r];
            D[4 + tt] = low ? hi_part[(tt * H + c) * kTM + r] : acc[tt][H + c];
          }
          const double v = oz_combine(D, ea, g.EB[j], kBeta, kS);
          g.C[i + j * g.ldc] = v;
          if (g.sym && i < j) g.C[j + i * g.ldc] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// D[t] summed over the K groups in 64-bit integers, then combined: C[i + j ldc]. One CTA of 8
// warps per 32 consecutive outputs i of one column j: warp w sums the groups w, w + 8, ...
// (lanes on consecutive i: coalesced rows of the partials), the 8 warps' sums are added in
// shared memory, and warp 0 combines. With sym (C = A^T A, product tiles below the diagonal
// skipped) only i <= j is combined and C[j + i ldc] receives the same value; the partials read
// then all come from computed tiles (i0 <= j puts rows i0 .. i0 + 31 in a tile that reaches
// column j).
__global__ void __launch_bounds__(256) k_oz_reduce(const int* __restrict__ part, int groups,
                                                   long long Mp, long long Np, long long M, int N,
                                                   const int* __restrict__ EA,
                                                   const int* __restrict__ EB,
                                                   double* __restrict__ C, long long ldc,
                                                   int sym) {
  __shared__ long long acc_sh[8][kS][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tiles_i = (M + 31) / 32;
  const long long i0 = (blockIdx.x % tiles_i) * 32, j = blockIdx.x / tiles_i;
  if (sym && i0 > j) return;
  const long long i = i0 + lane;  // < Mp: the padded rows of the partials exist
  int64_t D[kS];
#pragma unroll
  for (int d = 0; d < kS; ++d) D[d] = 0;
  for (int zz = warp; zz < groups; zz += 8)
#pragma unroll
    for (int d = 0; d < kS; ++d) D[d] += part[(((long long)zz * kS + d) * Np + j) * Mp + i];
#pragma unroll
  for (int d = 0; d < kS; ++d) acc_sh[warp][d][lane] = D[d];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int d = 0; d < kS; ++d) {
      long long t = 0;
      for (int w = 0; w < 8; ++w) t += acc_sh[w][d][lane];
      D[d] = t;
    }
    if (i < M && (!sym || i <= j)) {
      const double v = oz_combine(D, EA[i], EB[j], kBeta, kS);
      C[i + j * ldc] = v;
      if (sym && i < j) C[j + i * ldc] = v;
    }
  }
}

// max_r |X[r + c ld]| over r < d for every column c < n, as the bits of the FP64 value (for
// non-negative doubles the order of the bit patterns is the order of the values): grid (row
// chunks, columns); each CTA reduces its chunk and merges with an atomic maximum into mb[c],
// which the caller zeroes first
__global__ void k_oz_colmax(const double* __restrict__ X, long long ld, long long d, int n,
                            long long rows_per_cta, unsigned long long* __restrict__ mb) {
  const int c = blockIdx.y;
  const long long r0 = (long long)blockIdx.x * rows_per_cta;
  const long long r1 = min(d, r0 + rows_per_cta);
  double m = 0.0;
  if (c < n)
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) m = fmax(m, fabs(X[r + c * ld]));
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    if (m > 0.0) atomicMax(mb + c, (unsigned long long)__double_as_longlong(m));
  }
}

// E[c] = ceil(log2 max|x|) of column c (0 for zero columns and for the padding)
__global__ void k_oz_colexp_fin(const unsigned long long* __restrict__ mb, int ncols,
                                int* __restrict__ E) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncols) E[c] = oz_exponent(__longlong_as_double((long long)mb[c]));
}

// E[r] = ceil(log2 max_c |X[r + c ld]|) over c < n (one thread per row; 0 past d)
__global__ void k_oz_rowexp(const double* __restrict__ X, long long ld, long long d, int n,
                            long long rows_pad, int* __restrict__ E) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows_pad) return;
  double m = 0.0;
  if (r < d)
    for (int c = 0; c < n; ++c) m = fmax(m, fabs(X[r + c * ld]));
  E[r] = oz_exponent(m);
}

// The digits of one K value i of an octet, packed as they are stored: p[k][i / 2] holds digit k
// (BF16, exact: |a| <= 64) in its low half for even i and its high half for odd i. Packing as
// each value is split keeps 32 registers of digits per thread instead of 64 integers.
__device__ __forceinline__ void oz_pack_value(uint32_t (&p)[kS][4], int i, const int* a) {
#pragma unroll
  for (int k = 0; k < kS; ++k) {
    const uint32_t h = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)a[k]));
    if (i & 1)
      p[k][i >> 1] |= h << 16;
    else
      p[k][i >> 1] = h;
  }
}

// the 8 digits of one operand row's octet of K values into the layout with tiles of TR rows
__device__ __forceinline__ void oz_store_digits(unsigned char* out, int TR, long long ksteps,
                                                long long kstep, int kh, long long row,
                                                const uint32_t (&p)[kS][4]) {
  const long long tile = row / TR, rt = row - tile * TR;
#pragma unroll
  for (int k = 0; k < kS; ++k) {
    const size_t off = (((size_t)(tile * ksteps + kstep) * kS + k) * (TR / 8) + (rt >> 3)) * 256 +
                       kh * 128 + (rt & 7) * 16;
    *reinterpret_cast<uint4*>(out + off) = make_uint4(p[k][0], p[k][1], p[k][2], p[k][3]);
  }
}

// Operand rows = columns c of X (d x n, ld), K = rows r (Gram side; one exponent per column).
// One thread per (column, octet of 8 rows); consecutive threads take consecutive columns. The
// digits go to `out` in tiles of TR rows and, if out2 is not null, to out2 in tiles of TR2.
__global__ void k_oz_split_cols(const double* __restrict__ X, long long ld, long long d, int n,
                                const int* __restrict__ E, long long cols_pad, long long kpad,
                                unsigned char* __restrict__ out, int TR,
                                unsigned char* __restrict__ out2, int TR2, long long cols2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cols_pad * (kpad / 8)) return;
  const long long c = t % cols_pad, oct = t / cols_pad;
  const int e = E[c];
  uint32_t p[kS][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long r = oct * 8 + i;
    const double x = (c < n && r < d) ? X[r + c * ld] : 0.0;
    int a[kS];
    oz_slices(x, e, kBeta, kS, a);
    oz_pack_value(p, i, a);
  }
  oz_store_digits(out, TR, kpad / 16, oct >> 1, (int)(oct & 1), c, p);
  if (out2 && c < cols2) oz_store_digits(out2, TR2, kpad / 16, oct >> 1, (int)(oct & 1), c, p);
}

// Operand rows = rows r of X (d x n, ld), K = columns c (rotation side; one exponent per row).
// One thread per (row, octet of 8 columns); consecutive threads take consecutive rows.
__global__ void k_oz_split_rows(const double* __restrict__ X, long long ld, long long d, int n,
                                const int* __restrict__ E, long long rows_pad, long long kpad,
                                unsigned char* __restrict__ out, int TR) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows_pad * (kpad / 8)) return;
  const long long r = t % rows_pad, oct = t / rows_pad;
  const int e = E[r];
  uint32_t p[kS][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long c = oct * 8 + i;
    const double x = (r < d && c < n) ? X[r + c * ld] : 0.0;
    int a[kS];
    oz_slices(x, e, kBeta, kS, a);
    oz_pack_value(p, i, a);
  }
  oz_store_digits(out, TR, kpad / 16, oct >> 1, (int)(oct & 1), r, p);
}

long long rup(long long x, long long m) { return (x + m - 1) / m * m; }
size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct OzPlan {
  long long kpad, mpad, npad;  // K rows (multiple of 32); A-side rows (x128); B-side rows (x32)
  long long wins, groups;
  int wins_per_cta;
  size_t offEA, offEB, offMB, offA, offB, offP, total;
};

OzPlan plan(long long K, long long M, long long N, bool gram, bool same) {
  OzPlan p{};
  p.kpad = rup(K, kKC);
  p.mpad = rup(M, kTM);
  p.npad = rup(N, kTN);
  p.wins = (p.kpad + kWin - 1) / kWin;
  const long long tiles = (p.mpad / kTM) * (p.npad / kTN);
  long long groups = 1;
  if (gram) {
    groups = (2 * kSms + tiles - 1) / tiles;  // about two CTAs per SM
    if (groups > p.wins) groups = p.wins;
    const long long need = (p.wins + kMaxWinPerCta - 1) / kMaxWinPerCta;
    if (groups < need) groups = need;
  } else if (p.wins > kMaxWinPerCta) {
    groups = (p.wins + kMaxWinPerCta - 1) / kMaxWinPerCta;
  }
  p.wins_per_cta = (int)((p.wins + groups - 1) / groups);
  p.groups = (p.wins + p.wins_per_cta - 1) / p.wins_per_cta;
  size_t o = 0;
  p.offEA = o;
  o += al256((size_t)p.mpad * 4);
  p.offEB = o;
  o += al256((size_t)p.npad * 4);
  p.offMB = o;  // column maxima (bits), for the larger of the two sides
  o += al256((size_t)(p.mpad > p.npad ? p.mpad : p.npad) * 8);
  p.offA = o;
  o += al256((size_t)p.kpad * p.mpad * kS * 2);
  p.offB = o;  // the B side in tiles of 32 rows (also when A and B are one block)
  o += al256((size_t)p.kpad * p.npad * kS * 2);
  p.offP = o;
  o += p.groups > 1 ? al256((size_t)p.groups * kS * p.mpad * p.npad * 4) : 0;
  p.total = o;
  return p;
}

cudaError_t run(const OzPlan& p, const unsigned char* A, const unsigned char* B, const int* EA,
                const int* EB, long long M, int N, double* C, long long ldc, int* part,
                int* err, cudaStream_t st, bool sym, bool upper, bool n_fast) {
  cudaError_t e = cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmem);
  if (e != cudaSuccess) return e;
  OzArgs g{};
  g.A = A;
  g.B = B;
  g.ksteps = p.kpad / 16;
  g.kchunks = p.kpad / kKC;
  g.wins_per_cta = p.wins_per_cta;
  g.direct = p.groups == 1;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.EA = EA;
  g.EB = EB;
  g.part = part;
  g.Mp = p.mpad;
  g.Np = p.npad;
  g.err = err;
  g.sym = sym;
  g.upper = upper;
  const long long mtiles = p.mpad / kTM, ntiles = rup(N, kTN) / kTN;
  g.n_fast = n_fast && mtiles <= 65535;
  const dim3 grid = g.n_fast ? dim3((unsigned)ntiles, (unsigned)mtiles, (unsigned)p.groups)
                             : dim3((unsigned)mtiles, (unsigned)ntiles, (unsigned)p.groups);
  k_oz_mma<<<grid, kThreads, kSmem, st>>>(g);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (p.groups > 1) {
    const long long blocks = ((M + 31) / 32) * (long long)N;
    k_oz_reduce<<<(unsigned)blocks, 256, 0, st>>>(part, (int)p.groups, p.mpad, p.npad, M, N, EA,
                                                  EB, C, ldc, sym ? 1 : 0);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t col_exponents(const double* X, long long ld, long long d, int n, int cols_pad,
                          unsigned long long* mb, int* E, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(mb, 0, (size_t)cols_pad * 8, st);
  if (e != cudaSuccess) return e;
  // about 4 CTAs per SM in all, at least 2048 rows each
  long long chunks = (4 * kSms + n - 1) / (n > 0 ? n : 1);
  long long rows = (d + chunks - 1) / (chunks > 0 ? chunks : 1);
  if (rows < 2048) rows = 2048;
  chunks = (d + rows - 1) / rows;
  if (chunks < 1) chunks = 1;
  if (n > 0) {
    dim3 grid((unsigned)chunks, (unsigned)n);
    k_oz_colmax<<<grid, 256, 0, st>>>(X, ld, d, n, rows, mb);
  }
  k_oz_colexp_fin<<<(cols_pad + 255) / 256, 256, 0, st>>>(mb, cols_pad, E);
  return cudaGetLastError();
}

}  // namespace

size_t oz_gram_work_bytes(long long d, int na, int nb, bool same) {
  return plan(d, na, nb, true, same).total;
}

size_t oz_rotate_work_bytes(long long d, int k, int n) {
  return plan(k, d, n, false, false).total;
}

cudaError_t launch_oz_gram(const double* A, long long lda, const double* B, long long ldb,
                           long long d, int na, int nb, double* C, int ldc, void* work, int* err,
                           cudaStream_t st) {
  const bool same = A == B && lda == ldb && na == nb;
  const OzPlan p = plan(d, na, nb, true, same);
  unsigned char* w = static_cast<unsigned char*>(work);
  int* EA = reinterpret_cast<int*>(w + p.offEA);
  int* EB = same ? EA : reinterpret_cast<int*>(w + p.offEB);
  unsigned char* sa = w + p.offA;
  unsigned char* sb = w + p.offB;
  unsigned long long* mb = reinterpret_cast<unsigned long long*>(w + p.offMB);
  cudaError_t e0 = col_exponents(A, lda, d, na, (int)p.mpad, mb, EA, st);
  if (e0 != cudaSuccess) return e0;
  long long nt = p.mpad * (p.kpad / 8);
  // one split; with A and B one block it writes both layouts (tiles of 128 and of 32 rows)
  k_oz_split_cols<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(
      A, lda, d, na, EA, p.mpad, p.kpad, sa, kTM, same ? sb : nullptr, kTN, p.npad);
  if (!same) {
    if ((e0 = col_exponents(B, ldb, d, nb, (int)p.npad, mb, EB, st)) != cudaSuccess) return e0;
    nt = p.npad * (p.kpad / 8);
    k_oz_split_cols<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(B, ldb, d, nb, EB, p.npad,
                                                                  p.kpad, sb, kTN, nullptr, kTN, 0);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return run(p, sa, sb, EA, EB, na, nb, C, ldc, reinterpret_cast<int*>(w + p.offP), err, st,
             same, false, false);
}

cudaError_t launch_oz_rotate(const double* A, long long lda, const double* Q, int ldq,
                             long long d, int k, int n, double* C, long long ldc, void* work,
                             int* err, cudaStream_t st, bool upper) {
  const OzPlan p = plan(k, d, n, false, false);
  unsigned char* w = static_cast<unsigned char*>(work);
  int* EA = reinterpret_cast<int*>(w + p.offEA);
  int* EB = reinterpret_cast<int*>(w + p.offEB);
  unsigned char* sa = w + p.offA;
  unsigned char* sb = w + p.offB;
  k_oz_rowexp<<<(unsigned)((p.mpad + 255) / 256), 256, 0, st>>>(A, lda, d, k, p.mpad, EA);
  long long nt = p.mpad * (p.kpad / 8);
  k_oz_split_rows<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(A, lda, d, k, EA, p.mpad, p.kpad,
                                                                sa, kTM);
  cudaError_t e0 =
      col_exponents(Q, ldq, k, n, (int)p.npad, reinterpret_cast<unsigned long long*>(w + p.offMB),
                    EB, st);
  if (e0 != cudaSuccess) return e0;
  nt = p.npad * (p.kpad / 8);
  k_oz_split_cols<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(Q, ldq, k, n, EB, p.npad, p.kpad,
                                                                sb, kTN, nullptr, kTN, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the B-side tiles of one A tile run next to each other: the split A (d x k x 8 digits, far
  // above L2 at large d) then comes from HBM once instead of once per B-side tile
  return run(p, sa, sb, EA, EB, d, n, C, ldc, reinterpret_cast<int*>(w + p.offP), err, st,
             false, upper, true);
}

}  // namespace cs
