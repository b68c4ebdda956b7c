// FP32 angular kernel of H.X built from register-blocked contractions (see angular_gm.cuh).
// One CTA per (state tile of 8, radial node); 256 threads; chunks of 8 row pairs.
#include <cuda_runtime.h>

#include "angular_gm.cuh"
#include "cs_internal.h"
#include "hx_kernels.cuh"

namespace cs {

__global__ void __launch_bounds__(kGmThreads, 1) k_angular_gm(AngArgs<float> a, float* __restrict__ G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  angular_gm_block(a, G, blockIdx.y, blockIdx.x * kGmST, smem_raw);
}

cudaError_t launch_angular_gm(const AngArgs<float>& a, float* G, cudaStream_t stream) {
  const size_t smem = gm_smem_bytes(a.L, a.Q4, a.n_theta);
  if (!a.theta_pairs || !gm_eligible(a.L, a.Q4, a.n_theta))
    return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_angular_gm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.S + kGmST - 1) / kGmST, a.n_r);
  k_angular_gm<<<grid, kGmThreads, smem, stream>>>(a, G);
  return cudaGetLastError();
}

size_t build_theta_pairs(const std::vector<double>& theta, const std::vector<double>& trig,
                         int L, int Q4, int n_theta, std::vector<double>& out) {
  const GmShape g = gm_shape(L, Q4, n_theta);
  const int NP = (n_theta + 1) / 2;
  const size_t nth = gm_theta_pairs_elems(L, n_theta);
  out.assign(nth + gm_trig_elems(L, Q4), 0.0);
  for (int ch = 0; ch < g.nchunks; ++ch)
    for (int o = 0; o < g.RL; ++o)
      for (int p = 0; p < kGmRC; ++p) {
        const int jp = ch * kGmRC + p;
        if (jp < NP)
          out[((size_t)ch * (g.RL + 4) + o) * kGmRC + p] = theta[(size_t)jp * g.RL + o];
      }
  // phi tables in the kernel's shared-memory layouts. Tb[cos|sin][m < Lb][q < Qp] and
  // Tc[cos|sin][q < Qp + 1][mp < Lq], where mp lists the even m (padded to ne4), then the odd
  // m. Zero outside m < L, q < Q.
  const int Q = g.Q;
  double* Tb = out.data() + nth;
  double* Tc = Tb + 2 * (size_t)g.Lb * g.Qp;
  for (int c = 0; c < 2; ++c)
    for (int m = 0; m < g.Lb; ++m)
      for (int q = 0; q < g.Qp; ++q)
        Tb[((size_t)c * g.Lb + m) * g.Qp + q] =
            (m < L && q < Q) ? trig[((size_t)c * L + m) * Q + q] : 0.0;
  for (int c = 0; c < 2; ++c)
    for (int q = 0; q <= g.Qp; ++q)
      for (int mp = 0; mp < g.Lq; ++mp) {
        const int m = (mp < g.ne4) ? 2 * mp : 2 * (mp - g.ne4) + 1;
        Tc[((size_t)c * (g.Qp + 1) + q) * g.Lq + mp] =
            (m < L && q < Q) ? trig[((size_t)c * L + m) * Q + q] : 0.0;
      }
  return out.size();
}

}  // namespace cs
