/* include/cs_scf.h - self-consistent field pieces of libclusterspec (C ABI).
 *
 * The Kohn-Sham SCF cycle around the ChFSI eigensolver of cs.h:
 *   - electron density (Sec. 2.1 eq. density_expression, Sec. 2.2.5);
 *   - Hartree potential (Sec. 2.3.1 eqs. hartree_calc1, zeta_definition);
 *   - LDA exchange-correlation (Sec. 2.1: Slater exchange, Perdew-Zunger correlation);
 *   - Fermi-Dirac occupations with Brent's method (Sec. 3.4.1 eq. Fermi_constraint);
 *   - Anderson mixing of the effective potential (Sec. 3.4.1).
 *
 * Conventions:
 *   - Grid functions are DEVICE arrays of N_g = N_r N_theta N_phi doubles in the order
 *     [k][j][q] (the grid of cs_grid).
 *   - All arithmetic is FP64, except the Chebyshev filter inside cs_scf_step, which runs in the
 *     precision the caller picks.
 *   - Calls return a cs_status, with the message in cs_last_error(ctx).
 *   - Calls that read results back to the host are marked "Synchronising"; the others only
 *     enqueue work on `stream`.
 *   - The caller owns every buffer it passes. Objects created here own their internal buffers
 *     and free them in their _free call.
 */
#ifndef CLUSTERSPEC_CS_SCF_H
#define CLUSTERSPEC_CS_SCF_H

#include "cs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* States per inverse transform inside cs_density. */
#define CS_DENSITY_CHUNK 16
/* Largest Anderson history of cs_mixer_create. */
#define CS_MIXER_MAX_HISTORY 64
/* Largest number of integrals in one cs_grid_integrals call. */
#define CS_GRID_INTEGRALS_MAX 8

/* DEVICE workspace (bytes) of cs_density, cs_hartree and cs_grid_integrals on ctx. */
cs_status cs_scf_workspace_bytes(const cs_ctx* ctx, size_t* bytes);

/* rho[g] = 2 sum_s occ[s] psi_s(x_g)^2, with psi_s = B X[:, s] the inverse basis transform of
 * column s (eq. density_expression, spin-unpolarised; Sec. 2.2.5 transform method).
 * X: DEVICE FP64 d x n_s, leading dimension ld >= d. occ: DEVICE n_s doubles (0..1).
 * rho: DEVICE N_g doubles (written; no accumulation across calls). States are processed
 * CS_DENSITY_CHUNK at a time, and the sum over s runs in state order (deterministic). */
cs_status cs_density(cs_ctx* ctx, int n_s, const double* X, long long ld, const double* occ,
                     double* rho, void* work, cs_stream stream);

/* Hartree potential of a grid density (Sec. 2.3.1).
 * tau = B^T diag(W) rho are the density's coefficients in the orbitals' basis (the dualing
 * approximation), and V_H(x) = sum_lmn 4 pi/(2l+1) tau_lmn Y_lm(x) Z_ln(r) (eq.
 * hartree_calc1). Z_ln is evaluated in closed form:
 *   Z_ln(r) = (2l+1)/k_ln^2 R_ln(r) + sqrt(2/R^3) r^l R^(1-l) / k_ln,
 * which equals the Laplace-expansion integral of eq. zeta_definition exactly. The first term
 * is the Dirichlet eigenfunction solution; the second is the harmonic term that carries the
 * multipole moment to the boundary.
 * rho, vh: DEVICE N_g doubles; they must not overlap. */
cs_status cs_hartree(cs_ctx* ctx, const double* rho, double* vh, void* work, cs_stream stream);

/* Spin-unpolarised LDA at every grid point.
 *   eps_xc = Slater exchange -(3/4)(3 rho/pi)^(1/3) + Perdew-Zunger (1981) correlation in
 *            rs = (3/(4 pi rho))^(1/3).
 *   v_xc = d(rho eps_xc)/d rho.
 * Both are 0 where rho <= 0. rho, exc, vxc: DEVICE N_g doubles. exc or vxc may be NULL. */
cs_status cs_lda_xc(cs_ctx* ctx, const double* rho, double* exc, double* vxc,
                    cs_stream stream);

/* out[i] = sum_g W_g f[i][g] g[i][g] for i < n <= CS_GRID_INTEGRALS_MAX, with the grid
 * quadrature weights W (w_r w_theta 2 pi / N_phi).
 * f, g: HOST arrays of n DEVICE pointers to N_g doubles; a NULL g[i] means 1.
 * out: HOST n doubles. The reduction order is fixed (deterministic). Synchronising. */
cs_status cs_grid_integrals(cs_ctx* ctx, int n, const double* const* f,
                            const double* const* g, double* out, void* work, cs_stream stream);

/* Fermi-Dirac occupations f_i = 1/(1 + exp((lambda_i - mu)/kT)) with
 * sum_i f_i = n_electrons/2 (eq. Fermi_constraint). mu is found by Brent's method on the
 * bracket [min lambda - 60 kT - 1, max lambda + 60 kT + 1].
 * Also returns the electronic entropy S = -2 sum [f ln f + (1-f) ln(1-f)] (k_B = 1, two
 * spins). All arrays are HOST. Needs kT > 0 and 0 < n_electrons/2 < n; CS_ERR_ARG
 * otherwise. */
cs_status cs_fermi_occupations(int n, const double* lambda, double n_electrons, double kT,
                               double* occ, double* mu, double* entropy);

/* Anderson mixer of grid functions (Sec. 3.4.1).
 * Residual F_i = x_out,i - x_in,i. theta minimises
 *   || F_n - sum_j theta_j (F_n - F_{n-j}) ||_W   over the last m <= history iterates.
 * Then
 *   xbar = x_n - sum_j theta_j (x_n - x_{n-j}),
 *   Fbar = F_n - sum_j theta_j (F_n - F_{n-j}),
 *   x_next = xbar + beta Fbar.
 * The W-weighted Gram of the differences is formed on the device; its m x m normal
 * equations are solved on the host (Gaussian elimination with partial pivoting).
 * history = 0 gives linear mixing; at most CS_MIXER_MAX_HISTORY. The mixer owns device
 * copies of its history (2 (history + 1) N_g doubles).
 * cs_mixer_mix: x_in, x_out, x_next are DEVICE N_g doubles; x_next may alias x_in.
 * Synchronising (it reads the Gram back). */
typedef struct cs_mixer cs_mixer;
cs_status cs_mixer_create(cs_ctx* ctx, double beta, int history, cs_mixer** out);
cs_status cs_mixer_mix(cs_mixer* m, const double* x_in, const double* x_out, double* x_next,
                       cs_stream stream);
cs_status cs_mixer_reset(cs_mixer* m);
cs_status cs_mixer_free(cs_mixer* m);

/* SCF loop with potential mixing (Sec. 3.4.1), built from the calls above and the ChFSI of
 * cs.h. */
typedef struct {
  int n_s;                   /* states in the block */
  int n_want;                /* states whose residuals gate the first eigensolve */
  int degree;                /* Chebyshev degree of each ChFSI iteration */
  cs_precision filter_prec;  /* precision of the filter's H.X (CS_FP64, CS_FP32, ...) */
  double n_electrons;        /* electrons (two per fully occupied state) */
  double kT;                 /* Fermi-Dirac smearing temperature (Hartree), > 0 */
  double beta;               /* Anderson linear mixing parameter, (0, 1] */
  int history;               /* Anderson history, 0 .. CS_MIXER_MAX_HISTORY */
  double first_tol;          /* residual tolerance of the first ChFSI solve */
  int first_max_iter;        /* ChFSI iterations allowed in the first solve */
  int lanczos_k;             /* Lanczos steps of the filter's upper bound, 1 .. 64 */
  double e_ion;              /* constant added to the energy (ion-ion interaction) */
  int first_solver;          /* eigensolver of the first iteration: 0 ChFSI, 1 LOBPCG with the
                                Teter-Payne-Allan preconditioner (Sec. 3.1) */
} cs_scf_params;

typedef struct {
  int iteration;             /* 1-based SCF iteration just completed */
  int chfsi_iterations;      /* ChFSI iterations run in it */
  double energy;             /* free energy of the output density (Hartree) */
  double dE;                 /* energy - previous energy (0 on the first iteration) */
  double mu;                 /* Fermi level */
  double entropy;            /* electronic entropy (k_B = 1) */
  double band;               /* 2 sum f lambda */
  double e_hartree;          /* 1/2 int rho V_H[rho] */
  double e_xc;               /* int rho eps_xc[rho] */
  double max_resid;          /* largest Ritz residual of the block */
} cs_scf_report;

typedef struct cs_scf cs_scf;

/* Creates the SCF state. v_ext: the external (pseudo)potential on the grid; rho0: the
 * starting density; v0: the Lanczos start vector (d doubles). All are DEVICE arrays and are
 * copied. The first cs_scf_step sets v_in = v_ext + V_H[rho0] + v_xc[rho0]. */
cs_status cs_scf_create(cs_ctx* ctx, const cs_scf_params* p, const double* v_ext,
                        const double* rho0, const double* v0, cs_scf** out);
/* DEVICE workspace (bytes) of cs_scf_step. */
cs_status cs_scf_work_bytes(const cs_scf* s, size_t* bytes);

/* One SCF iteration on the block X (DEVICE FP64 d x n_s, ld).
 * 1. Set the potential v_in (cs_set_potential).
 * 2. Eigensolve. The first iteration runs cs_chfsi (first_solver 0) or cs_lobpcg
 *    (first_solver 1) to first_tol from the block as given. Later ones run one
 *    cs_chfsi_step with a = the previous largest Ritz value, a0 = the previous smallest, and
 *    b from lanczos_k Lanczos steps.
 * 3. Fermi-Dirac occupations, then the output density rho, V_H[rho] and the LDA.
 * 4. The free energy
 *      E = 2 sum f lambda - int rho (v_in - v_ext) + 1/2 int rho V_H + int rho eps_xc
 *          - kT S + e_ion.
 * 5. Anderson-mix v_in with v_out = v_ext + V_H + v_xc.
 * X receives the Ritz vectors. theta, resid: DEVICE n_s doubles. rep: HOST, filled.
 * Synchronising. CS_ERR_NOT_CONVERGED is not returned; max_resid reports the eigensolver's
 * state. */
cs_status cs_scf_step(cs_scf* s, double* X, long long ld, double* theta, double* resid,
                      void* work, cs_stream stream, cs_scf_report* rep);
/* Copies one of the SCF state's grid functions into out (DEVICE, N_g doubles), enqueued on
 * stream: which = 0 v_in (the next iteration's potential), 1 the last output density,
 * 2 its Hartree potential, 3 its eps_xc, 4 v_ext. CS_ERR_ARG for other values. */
cs_status cs_scf_grid(const cs_scf* s, int which, double* out, cs_stream stream);
/* HOST copy of the last occupations (n_s doubles). */
cs_status cs_scf_occupations(const cs_scf* s, double* occ);
cs_status cs_scf_free(cs_scf* s);

#ifdef __cplusplus
}
#endif

#endif /* CLUSTERSPEC_CS_SCF_H */
