// cs_apply_H_noalloc: H.X for callers that cannot allocate device memory when they call.
//
// cs_apply_H needs a caller-provided workspace for the radial-node intermediate G
// (N_r x (lmax+1)^2 x n_s elements). Some callers cannot provide one at the point of the
// call: for instance a process whose free device memory is already held by another
// allocator (a caching allocator that reserved it, so a fresh cudaMalloc fails), or a
// latency-critical loop that must not pay the implicit device-wide synchronisation of
// cudaMalloc/cudaFree. This variant takes its scratch from a fixed array compiled into
// the library (kScratchBytes below) instead, and allocates nothing itself. The context's
// tables are still created once, earlier, by cs_basis_init.
//
// Rules for users:
//   - The array holds kScratchBytes = 32 MiB on every GPU that loads this library, until
//     the process exits. Calls whose G does not fit are rejected with CS_ERR_ARG.
//   - The first call on each device looks the array's device address up
//     (cudaGetSymbolAddress) with that device current; make that first call before any
//     stream capture begins on that device. The address is kept for the process: after a
//     cudaDeviceReset of that device it is stale, and no later call may be made.
//   - Only CS_FP64 and CS_FP32 blocks are accepted (the split-BF16 and double-float modes
//     need staging buffers beyond G).
//   - The caller's current device is restored before the call returns.
//   - All calls on a device share the one array and it keeps the contents of the last
//     call. Two calls whose kernels overlap in time on the GPU (different streams, or
//     different host threads) race on it: serialise them.
//   - Nothing in the array has to start at zero: the radial synthesis writes every
//     element of G that the later kernels read.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "cs_internal.h"
#include "hx_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `dev` (which must be current); nullptr on error.
void* scratch_on_device(int dev, std::string& err) {
  if (dev < 0 || dev >= kMaxDevices) {
    err = "device index out of range for the static scratch table";
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress of the static scratch failed: ") +
            cudaGetErrorString(e);
      return nullptr;
    }
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

cs::DevTables<double>& tables_of(cs_ctx* c, const double*) { return c->d64; }
cs::DevTables<float>& tables_of(cs_ctx* c, const float*) { return c->d32; }

template <typename T>
cs_status run(cs_ctx* c, int n_s, const T* X, T* HX, long long ld, T* G, cudaStream_t st) {
  const cs::HostTables& H = c->host;
  cs::DevTables<T>& D = tables_of(c, X);
  cudaError_t e = cs::launch_radial_synth<T>(X, ld, G, D.rad, H.L, H.N, H.n_r, n_s, st);
  if (e == cudaSuccess) {
    c->launches += 1;
    // the same angular kernel as cs_apply_H (the FP32 one needs the transposed Legendre rows)
    cs::AngArgs<T> a{H.L,     H.n_r,   H.n_theta, H.n_phi, c->Q4, n_s,
                     D.theta, D.trig,  D.wv,      D.wkj,   D.theta_pairs};
    e = cs::launch_angular<T>(a, cs::ANG_FULL, G, nullptr, nullptr, st);
  }
  if (e == cudaSuccess) {
    c->launches += 1;
    cs::Epilogue<T> ep;
    ep.mode = cs::EP_APPLY;
    ep.out = HX;
    ep.X = X;
    ep.ld = ld;
    ep.ld_out = ld;
    ep.half_lambda = D.half_lambda;
    e = cs::launch_radial_anal<T>(G, D.rad, H.L, H.N, H.n_r, n_s, ep, st);
    if (e == cudaSuccess) c->launches += 1;
  }
  if (e != cudaSuccess) {
    c->err = std::string("cs_apply_H_noalloc launch: ") + cudaGetErrorString(e);
    return CS_ERR_CUDA;
  }
  return CS_OK;
}

}  // namespace

extern "C" cs_status cs_apply_H_noalloc(cs_ctx* c, int n_s, const void* X, void* HX,
                                        long long ld, cs_precision prec, cs_stream stream) {
  if (!c) return CS_ERR_ARG;
  if (!c->has_device) {
    c->err = "context has no device (created with device < 0)";
    return CS_ERR_STATE;
  }
  if (n_s < 1 || !X || !HX || ld < c->host.d || X == HX) {
    c->err = "cs_apply_H_noalloc: need n_s >= 1, non-NULL distinct X and HX, ld >= d";
    return CS_ERR_ARG;
  }
  if (prec != CS_FP64 && prec != CS_FP32) {
    c->err = "cs_apply_H_noalloc: precision must be CS_FP64 or CS_FP32";
    return CS_ERR_ARG;
  }
  if (!c->has_potential) {
    c->err = "cs_set_potential has not been called";
    return CS_ERR_STATE;
  }
  if (c->n_p > 0) {
    c->err = "cs_apply_H_noalloc does not apply projectors; use cs_apply_H";
    return CS_ERR_STATE;
  }
  const size_t elem = (prec == CS_FP64) ? 8 : 4;
  const size_t need = (size_t)c->host.n_r * c->host.L * c->host.L * (size_t)n_s * elem;
  if (need > kScratchBytes) {
    c->err = "cs_apply_H_noalloc: n_r*(lmax+1)^2*n_s*element size = " + std::to_string(need) +
             " bytes exceeds the static scratch of " + std::to_string(kScratchBytes) +
             " bytes; use fewer states per call or cs_apply_H";
    return CS_ERR_ARG;
  }
  int prev_dev = -1;
  cudaError_t e = cudaGetDevice(&prev_dev);
  if (e == cudaSuccess) e = cudaSetDevice(c->device);
  if (e != cudaSuccess) {
    c->err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    return CS_ERR_CUDA;
  }
  cs_status r = CS_ERR_CUDA;
  void* scratch = scratch_on_device(c->device, c->err);
  if (scratch) {
    cudaStream_t st = (cudaStream_t)stream;
    r = prec == CS_FP64
            ? run<double>(c, n_s, (const double*)X, (double*)HX, ld, (double*)scratch, st)
            : run<float>(c, n_s, (const float*)X, (float*)HX, ld, (float*)scratch, st);
  }
  if (prev_dev != c->device) cudaSetDevice(prev_dev);
  return r;
}
