// Internal declarations of libclusterspec (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cs.h"

namespace cs {

struct df64;  // double-float value (df64.cuh)

// ---------------------------------------------------------------- host tables (setup.cpp)
struct HostTables {
  double R = 0;
  int lmax = 0, L = 0, N = 0;
  long long d = 0;
  int n_r = 0, n_theta = 0, n_phi = 0, radial = 0;
  std::vector<double> z;        // [l][n]            Bessel zeros
  std::vector<double> r, w_r;   // [k]               radial nodes, weights (incl. r^2)
  std::vector<double> t, w_t;   // [j]               Gauss nodes in cos(theta), ascending
  std::vector<double> phi;      // [q]
  std::vector<double> rad;      // [l][k][n]         R_ln(r_k)
  std::vector<double> theta;    // [j][m][l-m]       Theta_lm(t_j) * (m>0 ? sqrt2 : 1), packed
  std::vector<double> half_lambda;  // [alpha]
};

// Builds every table on the host. Returns an empty string on success, else a message.
std::string build_host_tables(double R, int lmax, int nmax, const cs_quadrature& q,
                              HostTables& out);

// split-BF16 radial tables for the tensor-core path (tc_radial.cu); mode 0 synthesis, 1 analysis
void build_tc_tables(const HostTables& H, int mode, std::vector<uint16_t>& out, int& rows,
                     int& kpad);

// packed offset of (m, l) inside one theta row: sum_{m'<m} (L - m') + (l - m)
__host__ __device__ inline int theta_off(int L, int m) { return m * L - (m * (m - 1)) / 2; }
__host__ __device__ inline int theta_row_len(int L) { return L * (L + 1) / 2; }

// ---------------------------------------------------------------- device-side context
template <typename T>
struct DevTables {
  T* rad = nullptr;        // [l][k][n]
  T* theta = nullptr;      // [j][packed (m,l)], rows 0 .. ceil(n_theta/2)-1
  T* trig = nullptr;       // [2][lmax+1][Q4+1]: cos(m phi_q), sin(m phi_q), q <= Q4
  T* wv = nullptr;         // [k][j][q] W * V
  T* wkj = nullptr;        // [k][j] w_r w_t 2 pi / n_phi
  T* half_lambda = nullptr;// [alpha]
  T* pcoef = nullptr;      // [p][alpha] (d x n_p column-major)
  T* h = nullptr;          // [p] projector couplings
  T* theta_pairs = nullptr;// transposed Legendre rows of the register-blocked FP32 kernel
};

}  // namespace cs

struct cs_ctx {
  cs::HostTables host;
  int device = -1;
  bool has_device = false;
  bool has_potential = false;
  int n_p = 0;
  cs_precision rr_prec = CS_FP64;  // precision of the H.X that Rayleigh-Ritz projects
  cs_precision dense_prec = CS_FP64;  // Gram matrices and block rotations (FP64 or DF64)
  int Q4 = 0;              // floor(n_phi / 4): folded phi range q = 0 .. Q4
  cs::DevTables<double> d64;
  cs::DevTables<float> d32;
  cs::DevTables<cs::df64> ddf;  // double-float copies (CS_DF64)
  double* w_r_dev = nullptr; // radial weights (for forward transforms of grid data)
  double* hartree_tab = nullptr;  // k_ln = z_ln / R ([l][n]) then r_k / R ([k]) (scf.cu)
  double* grid_tab = nullptr;     // r_k, cos(theta_j), phi_q (learned.cu)
  void* tc_synth = nullptr;  // split-BF16 radial tables (tensor-core path)
  void* tc_anal = nullptr;
  void* tc_phi = nullptr;    // split-BF16 phi operands of the tensor-core angular kernel
  void* wide_tab = nullptr;  // split-BF16 Legendre and folded-trig operands of the wide block
  int tc_rows_synth = 0, tc_kpad_synth = 0, tc_rows_anal = 0, tc_kpad_anal = 0;
  void* kb_tabA = nullptr;   // split-BF16 projector operands (kb_tc.cu), set with the projectors
  void* kb_tabB = nullptr;
  int* dev_err = nullptr;    // device error word (bounded waits); 0 = ok
  std::string err;
  long long launches = 0;
  // measurement hooks (cs_profile_begin / cs_profile_end): class = kernel family
  // (0 radial synthesis, 1 angular, 2 radial analysis, 3 dense FP64, 4 projectors) + 5 when
  // the launch runs in FP32 / mixed precision, + 10 in double-float
  bool prof = false;
  struct ProfRec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_recs;
  std::vector<cudaEvent_t> event_pool;
};
