// Angular part of H.X (Sec. 2.2.2 eq. Ar_lm and the inverse transform, Sec. 2.2.4) with one
// warp per pair of mirrored theta rows, for the FMA pipes. Same arithmetic as k_angular in
// hx_kernels.cu (equatorial parity folding of the Legendre sums, four-angle folding of the
// phi sums), organised so that every shared-memory load feeds ST fused multiply-adds:
//   - a CTA owns radial node k and ST states; its warps take RC row pairs at a time;
//   - Legendre sums: each lane owns modes m and keeps the ST states in registers;
//   - phi sums and W V product: each lane owns folded angles q (all four mirror angles and
//     the ST states in registers), then writes the four folded quadrature inputs;
//   - phi quadrature: each lane owns modes m;
//   - Legendre quadrature: threads own (m, group of LG consecutive l), accumulating over
//     the chunk's row pairs into a shared-memory accumulator.
#include <cuda_runtime.h>

#include <type_traits>

#include "cs_internal.h"
#include "hx_kernels.cuh"
#include "angular_rp.cuh"

namespace cs {

template <typename T, int ST, int RC>
__global__ void __launch_bounds__(RC * 32) k_angular_rp(AngArgs<T> a, T* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  angular_rp_block<T, ST, RC>(a, G, blockIdx.y, blockIdx.x * ST, smem_raw);
}

template <typename T, int ST, int RC>
static cudaError_t launch_rp(const AngArgs<T>& a, T* G, cudaStream_t stream) {
  const int L = a.L, Q = a.Q4 + 1, rowlen = L * (L + 1) / 2;
  size_t smem = rp_smem_elems(L, Q, rowlen, ST, RC) * sizeof(T);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_angular_rp<T, ST, RC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.S + ST - 1) / ST, a.n_r);
  k_angular_rp<T, ST, RC><<<grid, RC * 32, smem, stream>>>(a, G);
  return cudaGetLastError();
}

// Variants: (ST, RC) = 0:(8,8) 1:(8,4) 2:(4,8) 3:(4,4) 4:(2,8) 5:(2,4). With variant < 0 the
// first variant of a measured preference order that fits in shared memory runs.
template <typename T>
cudaError_t launch_angular_rp(const AngArgs<T>& a, T* G, int variant, cudaStream_t stream) {
  const int L = a.L, Q = a.Q4 + 1, rowlen = L * (L + 1) / 2;
  const int st_rc[][2] = {{8, 8}, {8, 4}, {4, 8}, {4, 4}, {2, 8}, {2, 4}};
  auto fits = [&](int v) {
    return rp_smem_elems(L, Q, rowlen, st_rc[v][0], st_rc[v][1]) * sizeof(T) <= 227 * 1024;
  };
  if (variant < 0) {
    // measured on the 46128-function workload: (4,8) fastest in FP32 and FP64, (2,8) in
    // double-float (1.91 ms against 2.17 ms), whose per-thread state doubles the registers.
    // Where (4,8) does not fit (lmax 60 in FP32), (2,8) beats (4,4): 14.9 ms against 16.2 ms
    // on a 128-state chunk of the 357216-function workload.
    const int order_sp[] = {2, 0, 1, 4, 3, 5};
    const int order_df[] = {4, 2, 5, 3, 1, 0};
    const int* order = std::is_same<T, df64>::value ? order_df : order_sp;
    for (int i = 0; i < 6; ++i)
      if (fits(order[i])) {
        variant = order[i];
        break;
      }
    if (variant < 0) return cudaErrorInvalidConfiguration;
  }
  switch (variant) {
    case 0: return launch_rp<T, 8, 8>(a, G, stream);
    case 1: return launch_rp<T, 8, 4>(a, G, stream);
    case 2: return launch_rp<T, 4, 8>(a, G, stream);
    case 3: return launch_rp<T, 4, 4>(a, G, stream);
    case 4: return launch_rp<T, 2, 8>(a, G, stream);
    case 5: return launch_rp<T, 2, 4>(a, G, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
bool angular_rp_fits(int L, int Q4) {
  const int Q = Q4 + 1, rowlen = L * (L + 1) / 2;
  const int st_rc[][2] = {{8, 8}, {8, 4}, {4, 8}, {4, 4}, {2, 8}, {2, 4}};
  for (const auto& v : st_rc)
    if (rp_smem_elems(L, Q, rowlen, v[0], v[1]) * sizeof(T) <= 227 * 1024) return true;
  return false;
}
template bool angular_rp_fits<float>(int, int);
template bool angular_rp_fits<double>(int, int);
template bool angular_rp_fits<df64>(int, int);

template cudaError_t launch_angular_rp<float>(const AngArgs<float>&, float*, int, cudaStream_t);
template cudaError_t launch_angular_rp<double>(const AngArgs<double>&, double*, int, cudaStream_t);
template cudaError_t launch_angular_rp<df64>(const AngArgs<df64>&, df64*, int, cudaStream_t);

}  // namespace cs
