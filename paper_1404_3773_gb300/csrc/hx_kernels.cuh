// Launch interfaces of the H.X and dense linear-algebra kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

namespace cs {

struct df64;  // double-float value (df64.cuh)

enum { EP_PLAIN = 0, EP_APPLY = 1, EP_CHEB = 2 };
enum { ANG_FULL = 0, ANG_SYNTH = 1, ANG_ANAL = 2 };

// Epilogue of the radial analysis GEMM, for element (alpha, s):
//   EP_PLAIN : out = Z
//   EP_APPLY : out = 1/2 Lambda X + Z (+ kb)
//   EP_CHEB  : out = cA (1/2 Lambda X + Z (+ kb) (+ src_w[s] src) - cshift X) - cB Yprev
//              (Yprev may be out). The src term is the source of the residual form of the
//              filter: the Chebyshev recurrence run on the deviation D = p(H) X - X p(Theta)
//              of a block of Ritz vectors gains cA s_i(theta_s) R[:, s], R = H X - X Theta.
template <typename T>
struct Epilogue {
  int mode = EP_PLAIN;
  T* out = nullptr;
  const T* X = nullptr;
  const T* Yprev = nullptr;
  long long ld = 0;      // leading dimension of X
  long long ld_out = 0;  // leading dimension of out and Yprev
  const T* half_lambda = nullptr;
  const T* kb = nullptr;
  long long kb_ld = 0;
  const T* src = nullptr;    // d x S source block (residual form), or null
  const T* src_w = nullptr;  // S per-column weights of src
  long long src_ld = 0;
  T cA = T(0), cB = T(0), cshift = T(0);
};

template <typename T>
struct AngArgs {
  int L, n_r, n_theta, n_phi, Q4, S;
  const T* theta;  // [ceil(Nt/2)][L(L+1)/2]
  const T* trig;   // [2][L][Q4+1]
  const T* wv;     // [k][j][q]
  const T* wkj;    // [k][j] = w_r w_t 2 pi / Nphi (forward transforms of grid data)
  const T* theta_pairs = nullptr;  // FP32 only: Legendre rows by chunks of 8 mirrored pairs,
                                   // transposed ([chunk][packed (m,l) + 4][pair]); may be null
};

template <typename T>
int pick_states_per_cta(int L, int n_phi, int Q4);

template <typename T>
cudaError_t launch_angular(const AngArgs<T>& a, int mode, T* G, T* gout, const T* gin,
                           cudaStream_t stream);
// one-warp-per-row-pair variant of the ANG_FULL angular kernel (angular_rp.cu);
// variant -1 = first (states per CTA, row pairs per chunk) tile that fits shared memory
template <typename T>
cudaError_t launch_angular_rp(const AngArgs<T>& a, T* G, int variant, cudaStream_t stream);
// whether some row-pair tile fits in shared memory
template <typename T>
bool angular_rp_fits(int L, int Q4);

// three-pass double-float angular block for large lmax (angular_wide_df.cu): Legendre sums per
// m, folded phi transforms per grid row, Legendre quadrature per m, in blocks of 32 states
// through the double-float intermediate FA (angular_wide_df_work_bytes, one block); needs n_phi
// a multiple of 4. Taken where no row-pair tile fits, or with CS_ANGULAR_KERNEL=wide.
bool angular_wide_df_eligible(int L, int n_theta, int n_phi);
bool angular_wide_df_enabled(int L, int n_theta, int n_phi, int Q4);
size_t angular_wide_df_work_bytes(int L, int n_r, int n_theta);
cudaError_t launch_angular_wide_df(const AngArgs<df64>& a, df64* G, df64* FA,
                                   cudaStream_t stream);

// register-blocked FP32 angular kernel (angular_gm.cu); cudaErrorInvalidConfiguration when
// its tile does not fit in shared memory or the transposed Legendre table is missing
cudaError_t launch_angular_gm(const AngArgs<float>& a, float* G, cudaStream_t stream);
// builds the set-up table of the register-blocked kernel (host; returns the element count):
// the transposed Legendre table from the packed rows [ceil(n_theta/2)][L(L+1)/2], followed by
// the phi tables of trig ([cos|sin][m < L][q <= Q4]) in the kernel's shared-memory layouts
size_t build_theta_pairs(const std::vector<double>& theta, const std::vector<double>& trig,
                         int L, int Q4, int n_theta, std::vector<double>& out);

template <typename T>
cudaError_t launch_radial_synth(const T* X, long long ld, T* G, const T* rad, int L, int N,
                                int n_r, int S, cudaStream_t stream);
template <typename T>
cudaError_t launch_radial_anal(const T* G, const T* rad, int L, int N, int n_r, int S,
                               const Epilogue<T>& ep, cudaStream_t stream);

// ---------------------------------------------------------------- tensor-core radial GEMMs
struct HostTables;
// split-BF16 radial tables in the canonical tcgen05 operand layout (tc_radial.cu)
struct TcTables {
  const void* synth = nullptr;  // __nv_bfloat16, [l][k chunk][hi|lo][rows x 64]
  const void* anal = nullptr;
  int rows_synth = 0, kpad_synth = 0, rows_anal = 0, kpad_anal = 0;
};
// whether both radial tables fit the tensor-core kernels (radial dimensions <= 256)
bool tc_radial_fits(const HostTables& H);
cudaError_t launch_tc_radial_synth(const TcTables& tt, const HostTables& H, const float* X,
                                   long long ldx, float* G, int S, int* err,
                                   cudaStream_t stream);
cudaError_t launch_tc_radial_anal(const TcTables& tt, const HostTables& H, const float* G, int S,
                                  const Epilogue<float>& ep, int* err, cudaStream_t stream);

// angular block with the phi transforms on the tensor cores (angular_tc.cu, mixed precision):
// whether its tile fits, whether CS_ANGULAR_KERNEL leaves it enabled (unset or "tc"), the
// split-BF16 phi operands it copies to shared memory (uint16 BF16 bits), and the launch
// (cudaErrorInvalidConfiguration when the tile does not fit or a table is missing)
bool angular_tc_eligible(int L, int n_theta, int n_phi);
bool angular_tc_enabled();
void build_tc_phi_table(int L, int n_phi, std::vector<uint16_t>& out);
cudaError_t launch_angular_tc(const AngArgs<float>& a, const void* tphi, float* G, int* err,
                              cudaStream_t stream);

// three-pass tensor-core angular block for large lmax (angular_wide.cu): Legendre sums per m,
// folded phi transforms per grid row and Legendre quadrature per m, all split BF16 on tcgen05,
// through the FP32 intermediate FA (angular_wide_work_bytes); needs n_phi a multiple of 4
bool angular_wide_eligible(int L, int n_theta, int n_phi);
// the wide block is taken when eligible and the fused block is not, or when CS_ANGULAR_KERNEL
// starts with 'w'; any other non-empty CS_ANGULAR_KERNEL keeps it off
bool angular_wide_enabled(int L, int n_theta, int n_phi, bool fused_eligible);
size_t angular_wide_work_bytes(int L, int n_r, int n_theta, int S);
void build_wide_tables(const HostTables& H, std::vector<uint16_t>& out);
cudaError_t launch_angular_wide(const AngArgs<float>& a, const void* tab, float* G, float* FA,
                                int* err, cudaStream_t stream);

// ---------------------------------------------------------------- dense FP64 pieces
// C (na x nb, column-major, ldc) = A^T B, A: d x na (lda), B: d x nb (ldb), split over d
// into chunks whose partial products land in `partial` (gram_partial_elems doubles) and
// are then summed in a fixed order (deterministic).
// F = double or float (partials and sums in F).
size_t gram_partial_elems(long long d, int na, int nb);
template <typename F>
cudaError_t launch_gram(const F* A, long long lda, const F* B, long long ldb, long long d, int na,
                        int nb, F* C, int ldc, F* partial, cudaStream_t stream);
// C (d x n, ldc) = alpha * A (d x k, lda) * Q (k x n, ldq) + beta * C. A must not overlap C.
template <typename F>
cudaError_t launch_gemm_nn(const F* A, long long lda, const F* Q, int ldq, long long d, int k,
                           int n, double alpha, double beta, F* C, long long ldc,
                           cudaStream_t stream);
// the same two products on FP64 arrays with double-float arithmetic (FP32 pipe)
cudaError_t launch_gram_df(const double* A, long long lda, const double* B, long long ldb,
                           long long d, int na, int nb, double* C, int ldc, double* partial,
                           cudaStream_t stream);
cudaError_t launch_gemm_nn_df(const double* A, long long lda, const double* Q, int ldq,
                              long long d, int k, int n, double alpha, double beta, double* C,
                              long long ldc, cudaStream_t stream);
// y[p + s ld] *= h[p] for p < n_p, s < S
template <typename F>
cudaError_t launch_scale_rows(F* y, int n_p, int S, int ld, const F* h, cudaStream_t stream);
// From the Gram matrix M (n x n): U = D R^{-1}, D = diag(M)^(-1/2), D M D = R^T R.
// work: n*n + 2n doubles. status[0] = 0 ok, else 1 + index of the failing pivot.
cudaError_t launch_cholqr_factor(const double* M, int n, double* U, double* work, int* status,
                                 cudaStream_t stream);
// Symmetric eigensolve of sym(A) (n x n, lda = n): theta ascending, V (n x n) columns. An FP32
// solve (Householder tridiagonalisation, then bisection with inverse iteration, or QL where the
// bisection tiles do not fit in shared memory), Newton-Schulz re-orthonormalisation and
// Ogita-Aishima refinement in FP64, exact FP64 Jacobi inside clusters of near-equal values.
// work: 8n^2 + 3n + 4 doubles. status[0] = 1, or negative if a step did not converge.
// oz (oz_bytes), oz_err: optional slice-product workspace and its error word; with them the
// FP64 refinement products of large blocks run as slice products (launch_oz_gram/rotate).
cudaError_t launch_sym_eig(const double* A, int n, double* theta, double* V, double* work,
                              int* status, cudaStream_t stream, void* oz = nullptr,
                              size_t oz_bytes = 0, int* oz_err = nullptr);
// resid[i] = || HX[:, i] - theta[i] X[:, i] ||_2
cudaError_t launch_residuals(const double* X, long long ldx, const double* HX, long long ldh,
                             long long d, int n, const double* theta, double* resid,
                             cudaStream_t stream);
// y (d x n, ldy) = x (d x n, ldx) converted
cudaError_t launch_convert_f64_to_f32(const double* x, long long ldx, float* y, long long ldy,
                                      long long d, int n, cudaStream_t stream);
cudaError_t launch_convert_f32_to_f64(const float* x, long long ldx, double* y, long long ldy,
                                      long long d, int n, cudaStream_t stream);
// copy of a d x n block between leading dimensions
template <typename T>
cudaError_t launch_copy_block(const T* x, long long ldx, T* y, long long ldy, long long d,
                              int n, cudaStream_t stream);
// y = x / sqrt(*nrm2)  (length d)
cudaError_t launch_scale_inv_sqrt(const double* x, double* y, long long d, const double* nrm2,
                                  cudaStream_t stream);
// W V table: wv64[kj * n_phi + q] = wkj[kj] * v[kj * n_phi + q]; wv32 = (float) wv64;
// wvdf (optional) = wv64 split into double-float
cudaError_t launch_weighted_potential(const double* v, const double* wkj, int n_kj, int n_phi,
                                      double* wv64, float* wv32, df64* wvdf,
                                      cudaStream_t stream);
// double <-> double-float d x n blocks (in place allowed: same element size)
cudaError_t launch_to_df64(const double* x, long long ldx, df64* y, long long ldy, long long d,
                           int n, cudaStream_t stream);
cudaError_t launch_from_df64(const df64* x, long long ldx, double* y, long long ldy, long long d,
                             int n, cudaStream_t stream);
// Residual form of the Chebyshev filter (cheb_ritz.cu), T = double, float or df64:
// wd[i n + j] = s_i(theta_j), i = 0 .. m, the scaled filter polynomials on the Ritz values
// (c, e, sigma_1 = s1 as in the filter), and wt = wd rounded to T;
template <typename T>
cudaError_t launch_cheb_weights(const double* theta, int n, int m, double c, double e, double s1,
                                double* wd, T* wt, cudaStream_t stream);
// R = H X - X Theta and D1 = f1 R as T blocks with leading dimension d;
template <typename T>
cudaError_t launch_ritz_residual(const double* X, long long ldx, const double* HX, long long ldh,
                                 const double* theta, long long d, int n, double f1, T* R, T* D1,
                                 cudaStream_t stream);
// X <- X diag(sm) + D (D: T block with leading dimension d).
template <typename T>
cudaError_t launch_ritz_combine(double* X, long long ldx, const T* D, long long d, int n,
                                const double* sm, cudaStream_t stream);
// FP64 products from exact BF16 slice products on the tensor cores (ozaki_gemm.cu): the
// exactly rounded value of the truncated slice sum (beta 7, 8 digits). Workspace sizes first.
// Gram C (na x nb, ldc) = A^T B (A: d x na, B: d x nb); `same` when A and B are one block.
size_t oz_gram_work_bytes(long long d, int na, int nb, bool same);
cudaError_t launch_oz_gram(const double* A, long long lda, const double* B, long long ldb,
                           long long d, int na, int nb, double* C, int ldc, void* work, int* err,
                           cudaStream_t stream);
// Rotation C (d x n, ldc) = A (d x k, lda) Q (k x n, ldq). A must not overlap C. `upper`: Q is
// upper triangular (zeros stored below the diagonal), so each tile skips the zero rows.
size_t oz_rotate_work_bytes(long long d, int k, int n);
cudaError_t launch_oz_rotate(const double* A, long long lda, const double* Q, int ldq,
                             long long d, int k, int n, double* C, long long ldc, void* work,
                             int* err, cudaStream_t stream, bool upper = false);
// Lanczos tridiagonal T (k x k) from alpha[k] and the squared off-diagonals beta2[k-1]
cudaError_t launch_build_tridiag(const double* alpha, const double* beta2, int k, double* T,
                                 cudaStream_t stream);

}  // namespace cs
