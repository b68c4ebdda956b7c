// Measurement helper (not part of the method): sustained FP32 and FP64 fused multiply-add
// rates of the device, the denominators the benchmark rates its ALU-bound kernels against
// beside the nominal unit-count figures. Each thread runs 8 independent FMA chains (enough
// to cover the pipeline latency), on 4 CTAs of 256 threads per SM; the rate is flops over the
// CUDA-event time of one launch, the best of five.
#include <cuda_runtime.h>

#include "../../include/cs.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_stream(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)12345.678) out[blockIdx.x] = s;  // keeps the chains alive; never true here
}

template <typename T>
double time_fma(int nsm, int iters, T* out) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 4 * nsm;
  double best = 0.0;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0);
    k_fma_stream<T><<<blocks, 256>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * 256;
    if (rep > 0 && ms > 0.f) best = fmax(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace

extern "C" cs_status cs_measure_peaks(int cuda_device, double* fp32_tflops,
                                      double* fp64_tflops) {
  if (!fp32_tflops || !fp64_tflops) return CS_ERR_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(cuda_device) != cudaSuccess)
    return CS_ERR_CUDA;
  int nsm = 0;
  void* out = nullptr;
  cs_status st = CS_OK;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess ||
      cudaMalloc(&out, 8 * 4 * (size_t)nsm) != cudaSuccess) {
    st = CS_ERR_CUDA;
  } else {
    *fp32_tflops = time_fma<float>(nsm, 4096, static_cast<float*>(out));
    *fp64_tflops = time_fma<double>(nsm, 128, static_cast<double*>(out));
    if (cudaGetLastError() != cudaSuccess) st = CS_ERR_CUDA;
    cudaFree(out);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
