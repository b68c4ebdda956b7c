// Tensor-core Kleinman-Bylander projector products of the mixed-precision filter (kb_tc.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace cs {

// Tiling of the two products for d basis functions, n_p projectors and S states.
struct KbTcShape {
  long long d = 0;
  int n_p = 0, S = 0;
  int mtA = 0, kchA = 0;      // first product: 128-row projector tiles, 64-wide chunks of d
  long long mtB = 0;          // second product: 128-row tiles of d
  int kchB = 0;               // 64-wide chunks of n_p
  int stiles = 0;             // 128-state tiles
  int ksplit = 1, kper = 0;   // K split of the first product (CTAs along K, chunks per CTA)
  size_t tabA_bytes = 0, tabB_bytes = 0, xc_bytes = 0, wc_bytes = 0, part_bytes = 0;
};

KbTcShape kb_tc_shape(long long d, int n_p, int S);
// per-call scratch: split state block, split W, partial sums of the first product
size_t kb_tc_work_bytes(const KbTcShape& s);
// splits the FP64 projector coefficients (d x n_p, column-major, ld = d) into the two
// operand tables (tabA_bytes and tabB_bytes of kb_tc_shape(d, n_p, 1))
cudaError_t build_kb_tc_tables(const double* pcoef, long long d, int n_p, void* tabA, void* tabB,
                               cudaStream_t stream);
// Z (d x S, ldz) = P diag(h) P^T X (X: d x S FP32, ldx); 4 launches
cudaError_t launch_kb_tc(const void* tabA, const void* tabB, const KbTcShape& s, const float* X,
                         long long ldx, const float* h, float* Z, long long ldz, void* work,
                         int* err, cudaStream_t stream, int* launches);

}  // namespace cs
