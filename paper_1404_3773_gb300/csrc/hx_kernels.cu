// H.X kernels for FP64 and FP32 (FMA pipes). Sec. 2.2.4 eq. matvec_final:
//   H Y = 1/2 Lambda Y + forward( W V . inverse(Y) ) (+ projector pair)
// split into three launches per block of states:
//   k_radial_synth  : G[k][lm][s] = sum_n R_ln(r_k) X[alpha(l,m,n), s]         (eq. G_lmr)
//   k_angular       : per radial node k and a tile of states, inverse spherical harmonic
//                     transform (Legendre sums, phi sums), pointwise W V, forward
//                     transform (phi quadrature, Legendre quadrature), in place on G
//                     (eq. Ar_lm); nothing of the grid is written to memory
//   k_radial_anal   : Z[alpha, s] = sum_k R_ln(r_k) G'[k][lm][s]   (eq. Arlm_to_coeff, the
//                     weights sit in W V) with the epilogue 1/2 Lambda X + Z (+ KB) and,
//                     for the filter, the Chebyshev three-term update (Sec. 3.2.1).
// G layout: [k][lm][s] with lm = l^2 + l + m and S columns per row.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "cs_internal.h"
#include "df64.cuh"
#include "hx_kernels.cuh"
#include "hx_device.cuh"
#include "radial_gemm.cuh"

namespace cs {

// ------------------------------------------------------------------ radial GEMM tiles
template <typename T>
__global__ void __launch_bounds__(256) k_radial_synth(const T* __restrict__ X, long long ld,
                                                       T* __restrict__ G,
                                                       const T* __restrict__ rad, int L, int N,
                                                       int n_r, int S) {
  __shared__ T As[RBK][RBM + 1];
  __shared__ T Bs[RBK][RBN + 1];
  int l, c0;
  locate_l_tile(blockIdx.x, S, l, c0);
  radial_synth_tile<T>(X, ld, G, rad, L, N, n_r, S, l, c0, blockIdx.y * RBM, As, Bs);
}

template <typename T>
__global__ void __launch_bounds__(256) k_radial_anal(const T* __restrict__ G,
                                                      const T* __restrict__ rad, int L, int N,
                                                      int n_r, int S, Epilogue<T> ep) {
  __shared__ T As[RBK][RBM + 1];
  __shared__ T Bs[RBK][RBN + 1];
  int l, c0;
  locate_l_tile(blockIdx.x, S, l, c0);
  radial_anal_tile<T>(G, rad, L, N, n_r, S, ep, l, c0, blockIdx.y * RBM, As, Bs);
}

// FP32: register-blocked tiles (radial_gemm.cuh), RM rows per thread chosen from M
template <int MODE, int RM>
__global__ void __launch_bounds__(kRgThreads) k_radial_gemm(const float* __restrict__ X,
                                                             long long ldx, float* __restrict__ G,
                                                             const float* __restrict__ rad, int L,
                                                             int N, int n_r, int S,
                                                             Epilogue<float> ep) {
  __shared__ __align__(16) float sm[rg_smem_floats<RM>()];
  int l, c0;
  rg_locate(blockIdx.x, S, l, c0);
  radial_gemm_tile<MODE, RM>(X, ldx, G, rad, L, N, n_r, S, ep, l, c0, blockIdx.y * 16 * RM, sm);
}

template <int MODE>
static cudaError_t launch_radial_gemm(const float* X, long long ldx, float* G, const float* rad,
                                      int L, int N, int n_r, int S, const Epilogue<float>& ep,
                                      cudaStream_t stream) {
  const int M = (MODE == 0) ? n_r : N;
  const int rm = rg_rm(M);
  dim3 grid(rg_col_tiles(L, S), (M + 16 * rm - 1) / (16 * rm));
#define CS_RG_CASE(R)                                                                       \
  case R:                                                                                   \
    k_radial_gemm<MODE, R><<<grid, kRgThreads, 0, stream>>>(X, ldx, G, rad, L, N, n_r, S, ep); \
    break;
  switch (rm) {
    CS_RG_CASE(1)
    CS_RG_CASE(2)
    CS_RG_CASE(3)
    CS_RG_CASE(4)
    CS_RG_CASE(5)
    CS_RG_CASE(6)
    CS_RG_CASE(7)
    default:
      k_radial_gemm<MODE, 8><<<grid, kRgThreads, 0, stream>>>(X, ldx, G, rad, L, N, n_r, S, ep);
  }
#undef CS_RG_CASE
  return cudaGetLastError();
}

// ------------------------------------------------------------------ angular kernel
// One CTA: radial node k = blockIdx.y, states s0 .. s0+ST-1 (s0 = blockIdx.x * ST).
// Equatorial folding: t_j = -t_{Nt-1-j} and Theta_lm(-t) = (-1)^{l+m} Theta_lm(t), so the
// rows j and jb = Nt-1-j share one pass of Legendre sums (even/odd parts).
// Phi folding: with h = Nphi/2, the four angles phi_q, phi_{N-q}, phi_{h-q}, phi_{h+q}
// share cos/sin values up to signs (-1)^m, so sums run over q = 0 .. Nphi/4 only.
// MODE: ANG_FULL (synth, x W V, analysis, in place on G), ANG_SYNTH (synth -> grid
// [s][k][j][q]), ANG_ANAL (grid [s][k][j][q] x W -> analysis -> G).
template <typename T, int ST, int MODE>
__global__ void __launch_bounds__(256) k_angular(AngArgs<T> a, T* __restrict__ G,
                                                  T* __restrict__ grid_out,
                                                  const T* __restrict__ grid_in) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = a.L, lmax = L - 1, L2 = L * L, M2 = 2 * L - 1;
  const int Np = a.n_phi, h = Np / 2, Q4 = a.Q4, Q = Q4 + 1;
  const int Nt = a.n_theta, S = a.S;
  const int rowlen = L * (L + 1) / 2;
  T* Gs = reinterpret_cast<T*>(smem_raw);  // [L2][ST]
  T* Ga = Gs + (size_t)L2 * ST;            // [L2][ST]
  T* Fa = Ga + (size_t)L2 * ST;            // [2][M2][ST]
  T* Gb = Fa + (size_t)2 * M2 * ST;        // [2][Np][ST]
  T* Wb = Gb + (size_t)2 * Np * ST;        // [2][4][Q][ST]
  T* Ab = Wb + (size_t)8 * Q * ST;         // [2][M2][ST]
  T* tc = Ab + (size_t)2 * M2 * ST;        // [L][Q] cos(m phi_q)
  T* ts = tc + (size_t)L * Q;              // [L][Q] sin(m phi_q)
  T* th = ts + (size_t)L * Q;              // [rowlen]
  const int tid = threadIdx.x;
  const int k = blockIdx.y;
  const int s0 = blockIdx.x * ST;
  const int ns = min(ST, S - s0);

  for (int i = tid; i < 2 * L * Q; i += 256) tc[i] = a.trig[i];
  if (MODE != ANG_ANAL) {
    for (int i = tid; i < L2 * ST; i += 256) {
      int lm = i / ST, s = i - lm * ST;
      Gs[i] = (s < ns) ? G[((size_t)k * L2 + lm) * S + s0 + s] : T(0);
    }
  }
  if (MODE != ANG_SYNTH)
    for (int i = tid; i < L2 * ST; i += 256) Ga[i] = T(0);

  const int npairs = (Nt + 1) / 2;
  for (int jp = 0; jp < npairs; ++jp) {
    const int jrow[2] = {jp, Nt - 1 - jp};
    const bool single = (jrow[0] == jrow[1]);
    __syncthreads();  // previous pass done with th / buffers
    for (int i = tid; i < rowlen; i += 256) th[i] = a.theta[(size_t)jp * rowlen + i];
    __syncthreads();

    if (MODE != ANG_ANAL) {
      // (a2) Legendre sums, even/odd in l + |m|
      for (int it = tid; it < M2 * ST; it += 256) {
        int mi = it / ST, s = it - mi * ST;
        int m = mi - lmax, am = m < 0 ? -m : m;
        const T* tr = th + theta_off(L, am) - am;
        T E = T(0), O = T(0);
        for (int l = am; l <= lmax; l += 2) E = fma(tr[l], Gs[(l * l + l + m) * ST + s], E);
        for (int l = am + 1; l <= lmax; l += 2) O = fma(tr[l], Gs[(l * l + l + m) * ST + s], O);
        Fa[mi * ST + s] = E + O;
        Fa[(M2 + mi) * ST + s] = E - O;
      }
      __syncthreads();
      // (a3) phi sums over the folded range, (a4) times W V
      for (int it = tid; it < 2 * Q * ST; it += 256) {
        int row = it / (Q * ST);
        int rem = it - row * Q * ST;
        int q = rem / ST, s = rem - q * ST;
        const T* F = Fa + (size_t)row * M2 * ST;
        T Ee = F[lmax * ST + s], Eo = T(0), Oe = T(0), Oo = T(0);
        for (int m = 1; m <= lmax; m += 2) {
          Eo = fma(F[(lmax + m) * ST + s], tc[m * Q + q], Eo);
          Oo = fma(F[(lmax - m) * ST + s], ts[m * Q + q], Oo);
        }
        for (int m = 2; m <= lmax; m += 2) {
          Ee = fma(F[(lmax + m) * ST + s], tc[m * Q + q], Ee);
          Oe = fma(F[(lmax - m) * ST + s], ts[m * Q + q], Oe);
        }
        T v[4];
        int ix[4];
        int cnt = 0;
        ix[cnt] = q;
        v[cnt++] = (Ee + Eo) + (Oe + Oo);
        if (q > 0) {
          ix[cnt] = Np - q;
          v[cnt++] = (Ee + Eo) - (Oe + Oo);
        }
        if (2 * q != h) {
          ix[cnt] = h - q;
          v[cnt++] = (Ee - Eo) - (Oe - Oo);
          if (q > 0) {
            ix[cnt] = h + q;
            v[cnt++] = (Ee - Eo) + (Oe - Oo);
          }
        }
        const int jr = jrow[row];
        T* gout = Gb + (size_t)row * Np * ST;
        for (int c = 0; c < cnt; ++c) {
          if (MODE == ANG_FULL) {
            gout[ix[c] * ST + s] = a.wv[((size_t)k * Nt + jr) * Np + ix[c]] * v[c];
          } else if (s < ns && !(row == 1 && single)) {
            grid_out[((size_t)(s0 + s) * a.n_r + k) * Nt * Np + (size_t)jr * Np + ix[c]] = v[c];
          }
        }
      }
    } else {
      // grid input times quadrature weight W = w_r w_t 2 pi / Nphi
      for (int it = tid; it < 2 * Np * ST; it += 256) {
        int row = it / (Np * ST);
        int rem = it - row * Np * ST;
        int q = rem / ST, s = rem - q * ST;
        int jr = jrow[row];
        T v = T(0);
        if (s < ns)
          v = grid_in[((size_t)(s0 + s) * a.n_r + k) * Nt * Np + (size_t)jr * Np + q] *
              a.wkj[(size_t)k * Nt + jr];
        Gb[(size_t)row * Np * ST + q * ST + s] = v;
      }
    }
    if (MODE == ANG_SYNTH) continue;
    __syncthreads();
    // (a5) phi quadrature: fold the four angles into even/odd-in-m sums
    for (int it = tid; it < 2 * Q * ST; it += 256) {
      int row = it / (Q * ST);
      int rem = it - row * Q * ST;
      int q = rem / ST, s = rem - q * ST;
      const T* g = Gb + (size_t)row * Np * ST;
      T wq = (q == 0 || 2 * q == h) ? T(0.5) : T(1);
      T gq = g[q * ST + s];
      T gNq = g[((Np - q) % Np) * ST + s];
      T ghm = g[(h - q) * ST + s];
      T ghp = g[(h + q) * ST + s];
      T P = wq * (gq + gNq), Mm = wq * (gq - gNq);
      T P2 = wq * (ghm + ghp), M2v = wq * (ghm - ghp);
      T* w = Wb + (size_t)row * 4 * Q * ST;
      w[(0 * Q + q) * ST + s] = P + P2;    // cos, even m
      w[(1 * Q + q) * ST + s] = P - P2;    // cos, odd m
      w[(2 * Q + q) * ST + s] = Mm - M2v;  // sin, even m
      w[(3 * Q + q) * ST + s] = Mm + M2v;  // sin, odd m
    }
    __syncthreads();
    for (int it = tid; it < 2 * M2 * ST; it += 256) {
      int row = it / (M2 * ST);
      int rem = it - row * M2 * ST;
      int mi = rem / ST, s = rem - mi * ST;
      int m = mi - lmax, am = m < 0 ? -m : m;
      const T* w = Wb + (size_t)row * 4 * Q * ST;
      const T* src;
      const T* tab;
      if (m >= 0) {
        src = w + ((am & 1) ? 1 : 0) * Q * ST;
        tab = tc + am * Q;
      } else {
        src = w + ((am & 1) ? 3 : 2) * Q * ST;
        tab = ts + am * Q;
      }
      T acc = T(0);
      for (int q = 0; q <= Q4; ++q) acc = fma(tab[q], src[q * ST + s], acc);
      Ab[(size_t)row * M2 * ST + mi * ST + s] = acc;
    }
    __syncthreads();
    // (a6) Legendre quadrature, accumulated over row pairs
    for (int it = tid; it < L2 * ST; it += 256) {
      int lm = it / ST, s = it - lm * ST;
      int l = (int)sqrtf((float)lm);
      while (l * l > lm) --l;
      while ((l + 1) * (l + 1) <= lm) ++l;
      int m = lm - l * l - l, am = m < 0 ? -m : m;
      int mi = m + lmax;
      T v = Ab[mi * ST + s];
      if (!single) {
        T vb = Ab[(M2 + mi) * ST + s];
        v = ((l + am) & 1) ? v - vb : v + vb;
      }
      Ga[it] = fma(th[theta_off(L, am) + l - am], v, Ga[it]);
    }
  }
  if (MODE == ANG_SYNTH) return;
  __syncthreads();
  for (int i = tid; i < L2 * ST; i += 256) {
    int lm = i / ST, s = i - lm * ST;
    if (s < ns) G[((size_t)k * L2 + lm) * S + s0 + s] = Ga[i];
  }
}

// ------------------------------------------------------------------ launchers
template <typename T>
size_t angular_smem_bytes(int L, int n_phi, int Q4, int ST) {
  size_t L2 = (size_t)L * L, M2 = 2 * L - 1, Q = Q4 + 1;
  size_t elems = 2 * L2 * ST + 2 * M2 * ST + 2 * (size_t)n_phi * ST + 8 * Q * ST +
                 2 * M2 * ST + 2 * (size_t)L * Q + (size_t)L * (L + 1) / 2;
  return elems * sizeof(T);
}

template <typename T>
int pick_states_per_cta(int L, int n_phi, int Q4) {
  const size_t budget = 200 * 1024;
  for (int st : {16, 8, 4, 2, 1})
    if (sizeof(T) * st <= 128 && angular_smem_bytes<T>(L, n_phi, Q4, st) <= budget) return st;
  return 0;
}

template <typename T, int MODE>
static cudaError_t launch_angular_st(const AngArgs<T>& a, int st, T* G, T* gout, const T* gin,
                                     cudaStream_t stream) {
  size_t smem = angular_smem_bytes<T>(a.L, a.n_phi, a.Q4, st);
  dim3 grid((a.S + st - 1) / st, a.n_r);
  cudaError_t e = cudaSuccess;
#define CS_ANG_CASE(STV)                                                                   \
  case STV:                                                                                \
    e = cudaFuncSetAttribute(k_angular<T, STV, MODE>,                                      \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
    if (e != cudaSuccess) return e;                                                        \
    k_angular<T, STV, MODE><<<grid, 256, smem, stream>>>(a, G, gout, gin);                 \
    break;
  switch (st) {
    CS_ANG_CASE(16)
    CS_ANG_CASE(8)
    CS_ANG_CASE(4)
    CS_ANG_CASE(2)
    CS_ANG_CASE(1)
    default:
      return cudaErrorInvalidValue;
  }
#undef CS_ANG_CASE
  return cudaGetLastError();
}

// Which ANG_FULL kernel runs. FP32: the register-blocked kernel (angular_gm.cu) when its
// tile fits in shared memory, else the row-pair kernel (angular_rp.cu); FP64: the row-pair
// kernel; both fall back to the row-stream kernel above. CS_ANGULAR_KERNEL=gm|rp|rpN|stream
// overrides the choice (N = tile variant), for tuning.
static int angular_choice(int& variant) {
  variant = -1;
  const char* e = getenv("CS_ANGULAR_KERNEL");
  if (!e) return 0;
  if (e[0] == 's') return 3;
  if (e[0] == 'r' && e[1] == 'p') {
    variant = e[2] ? atoi(e + 2) : -1;
    return 2;
  }
  if (e[0] == 'g' && e[1] == 'm') {
    variant = e[2] ? atoi(e + 2) : -1;
    return 1;
  }
  return 0;
}

template <typename T>
cudaError_t launch_angular(const AngArgs<T>& a, int mode, T* G, T* gout, const T* gin,
                           cudaStream_t stream) {
  if (mode == ANG_FULL) {
    int variant;
    const int choice = angular_choice(variant);
    if constexpr (sizeof(T) == 4) {
      if (choice == 0 || choice == 1) {
        cudaError_t e = launch_angular_gm(a, G, stream);
        if (e != cudaErrorInvalidConfiguration) return e;
      }
    }
    if (choice != 3) {
      cudaError_t e = launch_angular_rp<T>(a, G, choice == 2 ? variant : -1, stream);
      if (e != cudaErrorInvalidConfiguration) return e;
    }
  }
  int st = pick_states_per_cta<T>(a.L, a.n_phi, a.Q4);
  if (st == 0) return cudaErrorInvalidConfiguration;
  if (mode == ANG_FULL) return launch_angular_st<T, ANG_FULL>(a, st, G, gout, gin, stream);
  if (mode == ANG_SYNTH) return launch_angular_st<T, ANG_SYNTH>(a, st, G, gout, gin, stream);
  return launch_angular_st<T, ANG_ANAL>(a, st, G, gout, gin, stream);
}

static int radial_col_tiles(int L, int S) {
  int t = 0;
  for (int l = 0; l < L; ++l) t += ((2 * l + 1) * S + RBN - 1) / RBN;
  return t;
}

template <typename T>
cudaError_t launch_radial_synth(const T* X, long long ld, T* G, const T* rad, int L, int N,
                                int n_r, int S, cudaStream_t stream) {
  if constexpr (std::is_same<T, float>::value)
    return launch_radial_gemm<0>(X, ld, G, rad, L, N, n_r, S, Epilogue<float>(), stream);
  dim3 grid(radial_col_tiles(L, S), (n_r + RBM - 1) / RBM);
  k_radial_synth<T><<<grid, 256, 0, stream>>>(X, ld, G, rad, L, N, n_r, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_radial_anal(const T* G, const T* rad, int L, int N, int n_r, int S,
                               const Epilogue<T>& ep, cudaStream_t stream) {
  if constexpr (std::is_same<T, float>::value)
    return launch_radial_gemm<1>(nullptr, 0, const_cast<float*>(G), rad, L, N, n_r, S, ep, stream);
  dim3 grid(radial_col_tiles(L, S), (N + RBM - 1) / RBM);
  k_radial_anal<T><<<grid, 256, 0, stream>>>(G, rad, L, N, n_r, S, ep);
  return cudaGetLastError();
}

template cudaError_t launch_angular<double>(const AngArgs<double>&, int, double*, double*,
                                            const double*, cudaStream_t);
template cudaError_t launch_angular<float>(const AngArgs<float>&, int, float*, float*,
                                           const float*, cudaStream_t);
template cudaError_t launch_radial_synth<double>(const double*, long long, double*,
                                                 const double*, int, int, int, int,
                                                 cudaStream_t);
template cudaError_t launch_radial_synth<float>(const float*, long long, float*, const float*,
                                                int, int, int, int, cudaStream_t);
template cudaError_t launch_radial_anal<double>(const double*, const double*, int, int, int,
                                                int, const Epilogue<double>&, cudaStream_t);
template cudaError_t launch_radial_anal<float>(const float*, const float*, int, int, int, int,
                                               const Epilogue<float>&, cudaStream_t);
template cudaError_t launch_angular<df64>(const AngArgs<df64>&, int, df64*, df64*, const df64*,
                                         cudaStream_t);
template cudaError_t launch_radial_synth<df64>(const df64*, long long, df64*, const df64*, int,
                                               int, int, int, cudaStream_t);
template cudaError_t launch_radial_anal<df64>(const df64*, const df64*, int, int, int, int,
                                              const Epilogue<df64>&, cudaStream_t);
template int pick_states_per_cta<df64>(int, int, int);
template int pick_states_per_cta<double>(int, int, int);
template int pick_states_per_cta<float>(int, int, int);

}  // namespace cs
