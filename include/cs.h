/*
 * cs.h -- C ABI of libclusterspec: the Chebyshev-filtered subspace iteration (ChFSI) hot
 * path of the spherical spectral Kohn-Sham method (Banerjee, Elliott, James, "A spectral
 * scheme for Kohn-Sham density functional theory of clusters"), on one GB300 (sm_103a).
 *
 * Problem statement the calls follow:
 *   basis     F_lmn = R_ln(r) Y_lm(theta, phi) on the ball |x| <= R, 0 <= l <= lmax,
 *             -l <= m <= l, 0 <= n < nmax; d = (lmax+1)^2 nmax functions (Sec. 2.2.1,
 *             eqs. eigfunction_1, spherical_bessel_1, spherical_harmonics_1). Real
 *             harmonics without the Condon-Shortley phase: Y_l0 = Theta_l0(cos theta),
 *             Y_lm = sqrt2 Theta_lm cos(m phi), Y_l,-m = sqrt2 Theta_lm sin(m phi), m > 0.
 *   index     alpha(l, m, n) = (l^2 + l + m) nmax + n  (0-based form of the footnote to
 *             eq. Hij_def).
 *   grid      N_r radial nodes with weights including r^2, N_theta Gauss points in
 *             cos(theta) in ascending order, N_phi uniform angles 2 pi q / N_phi
 *             (Sec. 2.2.2). Grid functions are [k][j][q] arrays, q fastest.
 *   operator  H = 1/2 diag(Lambda) + B^T diag(W V) B + P diag(h) P^T, B the synthesis
 *             matrix, W the quadrature weights, V the effective potential on the grid,
 *             P the projector coefficients (Sec. 2.2.4 eq. matvec_final, Sec. 2.3.2).
 *   filter    scaled Chebyshev filter of Sec. 3.2.1 (the cited Zhou-Saad recurrence).
 *
 * Conventions for every call:
 *   - Every call returns cs_status. No exception, exit or abort crosses the ABI.
 *     Arguments are checked before any launch (CS_ERR_ARG). cs_last_error(ctx) returns
 *     a message for the last failing call on that context.
 *   - Ownership: the caller owns every buffer it passes (host or device) and the library
 *     never frees one. A context owns its tables, allocated by cs_basis_init and
 *     freed by cs_basis_free.
 *   - Streams: cs_stream is a cudaStream_t (NULL = legacy default stream). All device
 *     work is enqueued on it. Calls return after enqueueing, except the ones documented
 *     as synchronising (they read FP64 scalars back).
 *   - Blocks X are column-major d x n_s with leading dimension ld >= d, one column per
 *     state, element type given by cs_precision (FP64: double; FP32: float).
 *   - A context is not thread-safe. It is bound to the CUDA device given at init.
 */
#ifndef CLUSTERSPEC_CS_H
#define CLUSTERSPEC_CS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_ctx cs_ctx;
typedef void* cs_stream; /* a cudaStream_t */

typedef enum {
  CS_OK = 0,
  CS_ERR_ARG = 1,           /* invalid argument (checked before any launch)          */
  CS_ERR_ALLOC = 2,         /* device or host allocation failed                      */
  CS_ERR_CUDA = 3,          /* a CUDA runtime call or a launch failed                */
  CS_ERR_STATE = 4,         /* call order violated (e.g. apply before set_potential)  */
  CS_ERR_CHOLESKY = 5,      /* Cholesky factorisation broke down (rank-deficient block) */
  CS_ERR_NOT_CONVERGED = 6, /* iteration limit reached before the tolerance           */
  CS_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up                     */
  CS_ERR_NUMERIC = 8        /* NaN or Inf detected in a result                        */
} cs_status;

typedef enum { CS_RADIAL_GAUSS_LEGENDRE = 0, CS_RADIAL_GAUSS_JACOBI_R2 = 1 } cs_radial_rule;

typedef struct {
  int n_r;     /* radial nodes                                        */
  int n_theta; /* Gauss points in cos(theta), > lmax                  */
  int n_phi;   /* uniform phi points, even, >= 2 lmax + 2             */
  int radial;  /* cs_radial_rule                                      */
} cs_quadrature;

typedef enum {
  CS_FP64 = 0,       /* FP64 storage and arithmetic                                      */
  CS_FP32 = 1,       /* FP32 storage and arithmetic (FP32 FMA pipe)                      */
  CS_MIXED_BF16 = 2  /* FP32 storage; the per-l radial contractions on the tensor cores
                        (tcgen05) with operands split into two BF16 terms (hi + lo, three
                        products, FP32 accumulation), and so are the two projector
                        products and, up to lmax 31, the angular block's phi synthesis and
                        phi quadrature; the Legendre sums and the recurrence in FP32.
                        Blocks are float.                                                */,
  CS_DF64 = 3        /* FP64 storage (blocks are double); H X computed in double-float
                        arithmetic on the FP32 pipe (each value an unevaluated sum of two
                        floats, about 48 significant bits; Dekker/Knuth error-free
                        transformations). On a GPU whose FP64 pipe runs at 1/64 of the FP32
                        rate this is several times faster than CS_FP64 at relative errors
                        near 1e-14. With projectors it is available for cs_apply_H and the
                        Rayleigh-Ritz apply only, and only with CS_FP64_SLICED dense
                        products (the projector term is then formed as exact slice products
                        and added in double-float); CS_ERR_STATE otherwise.               */,
  CS_FP64_SLICED = 4 /* dense products only (cs_set_dense_precision): FP64 Gram matrices and
                        rotations from exact products of 7-bit integer slices on the tensor
                        cores (Ozaki-Ogita-Oishi-Rump splitting, 8 slices per value, one
                        power of two per column or row); the result is the exactly rounded
                        value of the truncated slice sum, FP64-class (relative to |A|^T|B|
                        below 2^-53 d).                                                  */
} cs_precision;

/* ------------------------------------------------------------------ basis / context */

/* Build a context: Bessel zeros z_ln (Sec. 2.2.1 eq. laplacian_eigenvalue: Lambda_ln =
 * (z_ln/R)^2), radial table R_ln(r_k), normalised Legendre table Theta_lm(t_j), phi
 * twiddles, kinetic diagonal; uploads them to `cuda_device`. Host-side set-up, then
 * synchronous uploads. nmax = radial functions per l. Requirements: R > 0, 0 <= lmax,
 * nmax >= 1, n_theta > lmax, n_phi even and >= 2 lmax + 2, n_r >= 1.
 * On success *out owns device tables; free with cs_basis_free. */
cs_status cs_basis_init(double R, int lmax, int nmax, const cs_quadrature* q, int cuda_device,
                        cs_ctx** out);

/* Free a context and all tables it owns (synchronises its device). NULL is accepted. */
cs_status cs_basis_free(cs_ctx* ctx);

/* Sizes: d = (lmax+1)^2 nmax and the grid dimensions. Any pointer may be NULL. */
cs_status cs_basis_dims(const cs_ctx* ctx, long long* d, int* n_r, int* n_theta, int* n_phi);

/* Host copies (caller-allocated) of the grid: r[n_r], w_r[n_r] (weights include r^2),
 * t[n_theta] (= cos theta, ascending), w_t[n_theta], phi[n_phi]. Any pointer may be NULL. */
cs_status cs_grid(const cs_ctx* ctx, double* r, double* w_r, double* t, double* w_t,
                  double* phi);

/* Host copy of the kinetic diagonal 1/2 Lambda_alpha, length d (Sec. 2.2.4). */
cs_status cs_kinetic(const cs_ctx* ctx, double* half_lambda);

/* Host copy of the Bessel zeros z[l * nmax + n], (lmax+1) x nmax values. */
cs_status cs_bessel_zeros(const cs_ctx* ctx, double* z);

/* ------------------------------------------------------------------ operator set-up */

/* Set the effective potential V_eff (Sec. 2.2.3 eq. lin_eigen), given on the grid as a
 * DEVICE array of N_r * N_theta * N_phi doubles, layout [k][j][q]. The context stores
 * W * V (quadrature weights folded in) in FP64 and FP32. Enqueued on `stream`; the caller
 * may reuse v_grid once the stream has passed this call. */
cs_status cs_set_potential(cs_ctx* ctx, const double* v_grid, cs_stream stream);

/* Non-local Kleinman-Bylander part (Sec. 2.3.2): n_p rank-one projectors h_i p_i (x) p_i.
 * p_coef: DEVICE, d x n_p column-major (ld = d), the projector coefficients in this
 * basis (for grid values use cs_forward_transform first). h: HOST, n_p couplings.
 * The context copies both: FP64, FP32 and the split-BF16 operand tables of the tensor-core
 * products (4 + 4 + 4 + 4 bytes per coefficient, rounded up to 128-row x 64-column tiles),
 * then synchronises the stream. n_p = 0 removes the projectors. CS_ERR_ALLOC when the
 * tables do not fit in device memory. */
cs_status cs_set_projectors(cs_ctx* ctx, int n_p, const double* p_coef, const double* h,
                            cs_stream stream);

/* Forward basis transform (Sec. 2.2.2 eqs. Ar_lm, Arlm_to_coeff) of n grid functions:
 * g: DEVICE [n][N_r][N_theta][N_phi] doubles; coef: DEVICE d x n column-major with
 * leading dimension ld >= d; coef = B^T diag(W) g. work: DEVICE, at least
 * cs_workspace_bytes(ctx, n, CS_FP64) bytes. */
cs_status cs_forward_transform(cs_ctx* ctx, int n, const double* g, double* coef, long long ld,
                               void* work, cs_stream stream);

/* Inverse basis transform (Sec. 2.2.2 eq. G_lmr and the inverse spherical harmonic
 * transform): f[n][N_r][N_theta][N_phi] = (B coef)^T. Arguments as above. */
cs_status cs_inverse_transform(cs_ctx* ctx, int n, const double* coef, long long ld, double* f,
                               void* work, cs_stream stream);

/* Precision of the H X that Rayleigh-Ritz projects (cs_rayleigh_ritz, cs_chfsi_step,
 * cs_chfsi; Sec. 3.2.1). Default CS_FP64. With CS_FP32 or CS_MIXED_BF16 the block is rounded
 * to FP32, H is applied in that precision and the product is widened back; the projected
 * matrix X^T H X, its eigensolve, the rotations and the residual norms stay FP64. Residual
 * norms then level off near the reduced precision's H X error (about 1e-6 |H| for FP32 and
 * the split-BF16 mixed mode), so convergence thresholds should sit above that.
 * Workspaces must be sized (cs_workspace_bytes) after this call. CS_ERR_ARG for an unknown
 * precision. */
cs_status cs_set_rr_precision(cs_ctx* ctx, cs_precision prec);

/* Arithmetic of the tall-skinny Gram matrices (X^T X, X^T H X) and block rotations (X R^-1,
 * X Q, H X Q) of Cholesky-QR and Rayleigh-Ritz (Sec. 3.1.1, 3.2.1): CS_FP64 (default),
 * CS_DF64 (double-float on the FP32 pipe, FP64 storage, relative errors near 1e-14) or
 * CS_FP64_SLICED (exact integer-slice products on the tensor cores, rounded once; with it the
 * projector pair of every FP64 H.X is also taken as slice products, and so are the n x n
 * products of the eigensolve's FP64 refinement for blocks above 256 states). The small
 * factorisation, eigensolve and residual norms stay FP64. Workspaces must be sized
 * (cs_workspace_bytes) after this call. CS_ERR_ARG otherwise. */
cs_status cs_set_dense_precision(cs_ctx* ctx, cs_precision prec);

/* The dense steps' two products alone, in the context's dense precision (Sec. 3.2.1):
 * cs_dense_gram: C (na x nb, column-major, ldc >= na) = A^T B, A: d x na (lda), B: d x nb
 * (ldb), d the basis size; cs_dense_rotate: C (d x n, ldc >= d) = A Q, A: d x k (lda, must
 * not overlap C), Q: k x n (ldq >= k). All DEVICE FP64. work: cs_workspace_bytes(ctx,
 * max(na, nb) or max(k, n), CS_FP64) after cs_set_dense_precision. Enqueued on stream. */
cs_status cs_dense_gram(cs_ctx* ctx, int na, int nb, const double* A, long long lda,
                        const double* B, long long ldb, double* C, long long ldc, void* work,
                        cs_stream stream);
cs_status cs_dense_rotate(cs_ctx* ctx, int k, int n, const double* A, long long lda,
                          const double* Q, long long ldq, double* C, long long ldc, void* work,
                          cs_stream stream);

/* Device workspace (bytes) needed by cs_apply_H / cs_cheb_filter / transforms on n_s
 * columns at precision `prec`, and by cs_rayleigh_ritz / cs_chfsi (their FP64 needs are
 * included for prec = CS_FP64; for CS_FP32 the FP32 filter buffers are added). */
cs_status cs_workspace_bytes(const cs_ctx* ctx, int n_s, cs_precision prec, size_t* bytes);

/* ------------------------------------------------------------------ hot path */

/* HX = H X for a block of n_s states (Sec. 2.2.4 eq. matvec_final): per-l radial
 * synthesis GEMMs (eq. G_lmr), per-radial-node inverse and forward spherical harmonic
 * transforms with the pointwise W*V product, per-l radial analysis GEMMs (eq.
 * Arlm_to_coeff), plus 1/2 Lambda X and the projector pair. X, HX: DEVICE, d x n_s,
 * leading dimension ld, element type per prec; X and HX must not overlap.
 * Requires cs_set_potential first (CS_ERR_STATE otherwise). The tensor-core kernels of
 * CS_MIXED_BF16 bound every wait; one that expires leaves HX invalid, sets the context's
 * device error word and still returns CS_OK (the call does not synchronise): mixed-precision
 * callers read cs_device_error after synchronising (cs_cheb_filter likewise). */
cs_status cs_apply_H(cs_ctx* ctx, int n_s, const void* X, void* HX, long long ld,
                     cs_precision prec, void* work, cs_stream stream);

/* In place: X <- p_m(H) X = T_m((H - c)/e) X / T_m((a0 - c)/e), c = (a+b)/2,
 * e = (b-a)/2, by the scaled three-term recurrence (Sec. 3.2.1; degree m = `degree`
 * >= 1 H.X products). Requires a < b and a0 < a. X: DEVICE d x n_s, ld, type per prec. */
cs_status cs_cheb_filter(cs_ctx* ctx, int n_s, void* X, long long ld, int degree, double a,
                         double b, double a0, cs_precision prec, void* work,
                         cs_stream stream);

/* The same filter p_m(H) X for a block of Ritz vectors, in residual form (Sec. 3.2.1; the
 * algebra is this library's, the filter is the paper's). With R = H X - X Theta and s_i the
 * scaled filter polynomials evaluated at the Ritz values,
 *   p_m(H) X = X s_m(Theta) + D_m,  D_0 = 0,  D_1 = (sigma_1/e) R,
 *   D_{i+1} = (2 sigma_{i+1}/e) [(H - c) D_i + R s_i(Theta)] - sigma_i sigma_{i+1} D_{i-1},
 * an identity for any Theta. Only D meets H, in precision prec, so the rounding of an FP32 or
 * mixed H.X is relative to ||R||, not ||X||: as the Ritz pairs converge the filter's error
 * shrinks with them. It takes degree - 1 H.X products (D_1 needs none).
 * X: DEVICE FP64 d x n_s (ld), on entry the block, on exit p_m(H) X. HX: DEVICE FP64 H X
 * (ldh >= d), read only. theta: DEVICE n_s doubles. 1 <= degree <= 64, a0 < a < b as in
 * cs_cheb_filter. prec: CS_FP64, CS_DF64, CS_FP32 or CS_MIXED_BF16 (the arithmetic of the D
 * recurrence). work: cs_workspace_bytes(ctx, n_s, prec). */
cs_status cs_cheb_filter_ritz(cs_ctx* ctx, int n_s, double* X, long long ld, const double* HX,
                              long long ldh, const double* theta, int degree, double a, double b,
                              double a0, cs_precision prec, void* work, cs_stream stream);

/* Cholesky-QR with column scaling (Sec. 3.1.1, 3.2.1), applied twice: X <- X D R^{-1}
 * with D = diag(X^T X)^(-1/2), D X^T X D = R^T R. X: DEVICE FP64 d x n_s (ld).
 * Synchronising. CS_ERR_CHOLESKY if a pivot is not positive. */
cs_status cs_cholqr(cs_ctx* ctx, int n_s, double* X, long long ld, void* work,
                    cs_stream stream);

/* Rayleigh-Ritz on an orthonormal FP64 block (Sec. 3.2.1): HX = H X (precision set by
 * cs_set_rr_precision), Hs = sym(X^T H X) = Q Theta Q^T (device eigensolver), X <- X Q, and
 * the residual norms ||H x_i - theta_i x_i||_2. theta, resid: DEVICE n_s doubles (ascending
 * theta). If HX_out is not NULL it receives H X Q (DEVICE d x n_s, ld; must not overlap X).
 * Synchronising. */
cs_status cs_rayleigh_ritz(cs_ctx* ctx, int n_s, double* X, long long ld, double* theta,
                           double* resid, double* HX_out, void* work, cs_stream stream);

/* k-step Lanczos from the DEVICE vector v0 (length d, FP64, not modified): *b = largest
 * Ritz value + |beta_k| (upper bound of the spectrum for the filter), *theta_min =
 * smallest Ritz value. k <= 64. Synchronising. */
cs_status cs_lanczos_bound(cs_ctx* ctx, int k, const double* v0, double* b, double* theta_min,
                           void* work, cs_stream stream);

/* ChFSI loop (Sec. 3.2.1): Lanczos bounds from v0, then [filter (precision prec) ->
 * Cholesky-QR (FP64) -> Rayleigh-Ritz (FP64)] until the largest residual of the n_want
 * lowest Ritz pairs is <= tol or max_iter iterations. With prec CS_FP32 or CS_MIXED_BF16 (and
 * degree <= 64) every iteration after the first filters in residual form (as
 * cs_cheb_filter_ritz, from the previous iteration's Ritz values and H X), so its residuals
 * fall below the filter precision's level; FP64 and double-float filters stay plain. X: DEVICE FP64 d x n_s (ld), the
 * initial block on entry, the Ritz vectors on exit. theta, resid: DEVICE n_s doubles.
 * *iters receives the iteration count. First pass: a0 = smallest Lanczos Ritz value,
 * a = a0 + (b - a0)/10; later passes: a = largest Ritz value, a0 = smallest.
 * Synchronising. CS_ERR_NOT_CONVERGED if max_iter is reached (results still written). */
cs_status cs_chfsi(cs_ctx* ctx, int n_s, int n_want, double* X, long long ld, int degree,
                   double tol, int max_iter, cs_precision prec, const double* v0,
                   double* theta, double* resid, int* iters, void* work, cs_stream stream);

/* One ChFSI iteration (Sec. 3.2.1) with given filter bounds: X <- p_m(H) X (precision prec),
 * Cholesky-QR (FP64), Rayleigh-Ritz (FP64) with residual norms. X: DEVICE FP64 d x n_s
 * (ld), orthonormal or not on entry, Ritz vectors on exit. theta, resid: DEVICE n_s
 * doubles. Synchronising (reads the factorisation status back). */
cs_status cs_chfsi_step(cs_ctx* ctx, int n_s, double* X, long long ld, int degree, double a,
                        double b, double a0, cs_precision prec, double* theta, double* resid,
                        void* work, cs_stream stream);

/* One ChFSI iteration (Sec. 3.2.1) whose filter takes the residual form (cs_cheb_filter_ritz):
 * X, HX, theta in: Ritz vectors (DEVICE FP64 d x n_s, ld), their H X (same shape and ld) and
 * Ritz values (DEVICE n_s); out: the next Ritz vectors, their H X and Ritz values, and resid
 * (DEVICE n_s) the residual norms. Cholesky-QR and Rayleigh-Ritz as in cs_chfsi_step; the
 * outgoing H X is Rayleigh-Ritz's (cs_set_rr_precision) rotated by Q. 1 <= degree <= 64.
 * Synchronising. */
cs_status cs_chfsi_step_ritz(cs_ctx* ctx, int n_s, double* X, double* HX, long long ld,
                             int degree, double a, double b, double a0, cs_precision prec,
                             double* theta, double* resid, void* work, cs_stream stream);

/* LOBPCG (Sec. 3.1) with the diagonal Teter-Payne-Allan preconditioner (Sec. 3.1.2), FP64:
 * the lowest n_s eigenpairs of H from the block X (DEVICE FP64 d x n_s, ld; Ritz vectors on
 * exit). Each iteration runs Rayleigh-Ritz on [X, W, P]:
 *   - W: the preconditioned residuals of the columns whose residual is above tol (soft
 *     locking), made orthogonal to X and orthonormalised (Cholesky-QR twice, column scaling);
 *   - P: the previous search directions, orthonormalised.
 * Convergence: the largest residual norm of the n_want lowest pairs <= tol.
 * A Cholesky breakdown discards the iteration and restarts from the current Ritz vectors (W
 * and P dropped).
 * precondition = 0 switches the preconditioner off. The preconditioner scales coefficient
 * alpha of a residual column y by
 *   (27 + 18g + 12g^2 + 8g^3) / (27 + 18g + 12g^2 + 8g^3 + 16g^4),
 *   g = Lambda_alpha / (1/2 sum Lambda y^2 / sum y^2).
 * theta, resid: DEVICE n_s doubles. *iters receives the iteration count and *restarts the
 * restarts (either may be NULL). work: DEVICE, cs_lobpcg_workspace_bytes(ctx, n_s) bytes.
 * Synchronising. CS_ERR_NOT_CONVERGED after max_iter iterations (results written);
 * CS_ERR_CHOLESKY if the starting block is rank deficient. */
cs_status cs_lobpcg_workspace_bytes(const cs_ctx* ctx, int n_s, size_t* bytes);
cs_status cs_lobpcg(cs_ctx* ctx, int n_s, int n_want, double* X, long long ld, double tol,
                    int max_iter, int precondition, double* theta, double* resid, int* iters,
                    int* restarts, void* work, cs_stream stream);

/* Measurement hooks: between cs_profile_begin and cs_profile_end the library records a
 * CUDA event pair on the launching stream around every kernel it launches on ctx.
 * cs_profile_end synchronises, and writes per kernel class the summed device time
 * (ms[CS_PROFILE_CLASSES]) and the launch count (launches[CS_PROFILE_CLASSES]). Class =
 * family + 5 for launches in FP32 / mixed precision, + 10 in double-float (FP64 launches:
 * family alone); families:
 * 0 radial synthesis GEMMs, 1 angular transforms (per radial node), 2 radial analysis GEMMs
 * with the fused epilogue, 3 dense FP64 linear algebra and conversions, 4 Kleinman-Bylander
 * projector products. */
#define CS_PROFILE_CLASSES 15
cs_status cs_profile_begin(cs_ctx* ctx);
cs_status cs_profile_end(cs_ctx* ctx, double* ms, long long* launches);

/* H X like cs_apply_H, for callers that cannot allocate device memory when they call (for
 * example when another allocator already holds the free device memory, or when a loop must
 * not take the device-wide synchronisation of cudaMalloc/cudaFree). It needs no workspace:
 * its scratch is a 32 MiB array compiled into the library, present on every GPU that loads
 * the library until the process exits; it calls no allocation routine. The paper has no
 * counterpart; this is a deployment variant of the same H.X kernels.
 * Limits and rules: prec must be CS_FP64 or CS_FP32 (CS_ERR_ARG otherwise); N_r (lmax+1)^2
 * n_s x element size must be <= 32 MiB (else CS_ERR_ARG); no projectors (CS_ERR_STATE if
 * set); the first call on a device looks up the array's device address and keeps it, so make
 * that call before any stream capture on that device, and make no call on a device after a
 * cudaDeviceReset of it; all calls on a device share the array (it keeps the last call's
 * contents; nothing in it must start at zero), so calls that overlap on the GPU race and must
 * be serialised. The caller's current device is restored on return. Other arguments as
 * cs_apply_H without `work`. */
cs_status cs_apply_H_noalloc(cs_ctx* ctx, int n_s, const void* X, void* HX, long long ld,
                             cs_precision prec, cs_stream stream);

/* ------------------------------------------------------------------ batched filter */

/* Many independent clusters (contexts of uneven lmax, N, grid and state count) filtered
 * together, FP32 blocks (Sec. 3.2.1 filter, Sec. 2.2.4 H.X per cluster). The radial,
 * angular and radial-analysis tiles of every cluster form one work list per Chebyshev step,
 * run either by one persistent launch per step (bounded waits between the stages of a
 * cluster) or staged, one launch per (stage, tile shape) group (see cs_batch_tune_times);
 * the filter is captured once into a CUDA graph and replayed. Every cluster's result is
 * bitwise equal to cs_cheb_filter on that cluster alone (CS_FP32). All contexts must be on one
 * device, have a potential and no projectors. n_s[i] states for cluster i; degree fixed per
 * batch. */
typedef struct cs_batch cs_batch;
cs_status cs_batch_create(int n, cs_ctx* const* ctxs, const int* n_s, int degree,
                          cs_batch** out);
cs_status cs_batch_free(cs_batch* batch);
/* DEVICE workspace needed by cs_batch_cheb_filter and cs_batch_tune (bytes). */
cs_status cs_batch_workspace_bytes(const cs_batch* batch, size_t* bytes);
/* X[i]: DEVICE float block of cluster i (d_i x n_s[i], leading dimension ld[i]), filtered in
 * place with bounds (a[i], b[i], a0[i]) (HOST arrays). Enqueued on `stream`; the first call
 * (or a call after cs_batch_tune) captures the graph, so make it outside stream capture. */
cs_status cs_batch_cheb_filter(cs_batch* batch, float* const* X, const long long* ld,
                               const double* a, const double* b, const double* a0, void* work,
                               cs_stream stream);
/* Autotuner: times one filter per variant (launch form x angular tile, see
 * cs_batch_tune_times) on these blocks and keeps the fastest; X is restored afterwards.
 * Synchronising. *chosen = variant index, *best_ms = its filter time. */
cs_status cs_batch_tune(cs_batch* batch, float* const* X, const long long* ld, const double* a,
                        const double* b, const double* a0, void* work, cs_stream stream,
                        int* chosen, float* best_ms);

/* Filter time (ms) of each variant in the last cs_batch_tune (-1 where not timed), for n
 * variants: 0 .. 2 one persistent launch per Chebyshev step with row-pair angular tiles of 4, 8
 * and 2 states; 3 one launch per (stage, tile shape) group of items; 4 every cluster's filter
 * as the single-cluster kernels of cs_cheb_filter, the clusters dealt (largest first, to the
 * least loaded) over 8 parallel branches of the graph, so that small clusters overlap. */
cs_status cs_batch_tune_times(const cs_batch* batch, float* ms, int n);
/* Selects a variant (as numbered above) without timing; the next filter call recaptures its
 * graph. CS_ERR_ARG for an unknown variant or one that does not fit in shared memory. */
cs_status cs_batch_set_variant(cs_batch* batch, int variant);
/* Precision of the batch: CS_FP32 (default) or CS_MIXED_BF16 (the split-BF16 tensor-core
 * kernels of cs_cheb_filter's mixed mode; blocks stay float). The mixed precision runs variant
 * 4 only, and every cluster's result is then bitwise equal to cs_cheb_filter on that cluster
 * alone in CS_MIXED_BF16. The next filter call recaptures its graph. */
cs_status cs_batch_set_precision(cs_batch* batch, cs_precision prec);
const char* cs_batch_last_error(const cs_batch* batch);

/* Device error word of the context (synchronising): 0 if no kernel reported a problem, else
 * the code of the first bounded wait that expired (tensor-core path). Reading clears it. A
 * non-zero word is also reported as CS_ERR_TIMEOUT by the next synchronising call. */
cs_status cs_device_error(cs_ctx* ctx, int* code);

/* Last error message of the context (static storage inside ctx; "" if none). A NULL ctx
 * returns the message of the last failed cs_basis_init on this thread. */
const char* cs_last_error(const cs_ctx* ctx);

/* Measurement helper for roofline denominators (the paper has no counterpart): the
 * sustained FP32 and FP64 fused multiply-add rates of device `cuda_device` in TFLOP/s (8
 * independent FMA chains per thread, 4 CTAs of 256 threads per SM, best of five timed
 * launches). Synchronising; restores the caller's current device. */
cs_status cs_measure_peaks(int cuda_device, double* fp32_tflops, double* fp64_tflops);

/* Number of kernels this library has launched on `ctx` since it was created. */
long long cs_launch_count(const cs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CLUSTERSPEC_CS_H */
