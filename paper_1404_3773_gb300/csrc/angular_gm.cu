// FP32 angular kernel of H.X built from register-blocked contractions (see angular_gm.cuh).
// One CTA per (state tile of 8, radial node); 256 threads; chunks of 8 (or 4) row pairs.
#include <cuda_runtime.h>

#include "angular_gm.cuh"
#include "cs_internal.h"
#include "hx_kernels.cuh"

namespace cs {

template <int ST, int RC>
__global__ void __launch_bounds__(kGmThreads) k_angular_gm(AngArgs<float> a, float* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  angular_gm_block<ST, RC>(a, G, blockIdx.y, blockIdx.x * ST, smem_raw);
}

template <int ST, int RC>
static cudaError_t launch_gm(const AngArgs<float>& a, float* G, cudaStream_t stream) {
  const size_t smem = gm_smem_bytes(a.L, a.Q4, ST, RC);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_angular_gm<ST, RC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.S + ST - 1) / ST, a.n_r);
  k_angular_gm<ST, RC><<<grid, kGmThreads, smem, stream>>>(a, G);
  return cudaGetLastError();
}

// 8 states per CTA with 8 row pairs per chunk, else 4 row pairs; cudaErrorInvalidConfiguration
// when neither fits in shared memory (the caller then takes another angular kernel)
cudaError_t launch_angular_gm(const AngArgs<float>& a, float* G, int variant, cudaStream_t stream) {
  if (variant <= 0 && gm_smem_bytes(a.L, a.Q4, 8, 8) <= 227 * 1024) return launch_gm<8, 8>(a, G, stream);
  if (variant <= 1 && gm_smem_bytes(a.L, a.Q4, 8, 4) <= 227 * 1024) return launch_gm<8, 4>(a, G, stream);
  return cudaErrorInvalidConfiguration;
}

}  // namespace cs
