/* include/cs_learned.h - learned initial SCF density of libclusterspec (C ABI).
 *
 * A small network predicts, from the neighbourhood of each atom, a correction to the SCF
 * starting density, so that the SCF of Sec. 3.4.1 starts closer to its fixed point.
 *
 * Per atom:
 *   - a radial descriptor D_ak = sum_{b != a} exp(-(r_ab - mu_k)^2 / (2 w^2));
 *   - an atom-centred correction sum_j c_aj phi_j(|x - a|), with the unit-integral Gaussians
 *     phi_j(r) = (2 pi s_j^2)^(-3/2) exp(-r^2 / (2 s_j^2)).
 * A tanh multilayer perceptron maps D_a to c_a. It is trained on coefficients fitted, by
 * quadrature-weighted least squares, to converged densities that the solver produced.
 * Training uses the mean squared error and Adam (Kingma & Ba 2015).
 *
 * Layouts:
 *   - The network's activations are FP32 column-major matrices with one row per atom
 *     (X[a + i n], n rows).
 *   - Each weight matrix W_l is column-major n_in x n_out, stored as W_l[i + j n_in].
 *   - Parameters are W_1, b_1, W_2, b_2, ... concatenated.
 *   - Grid functions are DEVICE FP64 arrays of N_g values in cs_grid order.
 * Calls marked "Synchronising" read results back to the host. */
#ifndef CLUSTERSPEC_CS_LEARNED_H
#define CLUSTERSPEC_CS_LEARNED_H

#include "cs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* HOST: descriptors out[a k] (n_atoms x n_mu, row-major) of the atoms (n_atoms x 3 bohr). */
cs_status cs_atom_descriptors(int n_atoms, const double* atoms, int n_mu, const double* mu,
                              double width, double* out);

/* rho[g] += sum_a sum_j coef[a n_basis + j] phi_j(|x_g - atoms[a]|) on ctx's grid.
 * atoms, sigmas, coef are HOST; rho is DEVICE N_g doubles. */
cs_status cs_atom_density(cs_ctx* ctx, int n_atoms, const double* atoms, int n_basis,
                          const double* sigmas, const double* coef, double* rho,
                          cs_stream stream);

/* Least-squares fit of a grid function by the same expansion:
 *   coef = argmin sum_g W_g (sum_{a,j} coef_aj phi_j(|x_g - a|) - target_g)^2
 *          + ridge tr(M)/n_c |coef|^2.
 * The normal equations M = A^T W A and A^T W target are accumulated on the device, in chunks
 * of grid points; the n_c = n_atoms n_basis system is solved on the host by Cholesky.
 * target: DEVICE N_g doubles. coef: HOST n_atoms x n_basis (out). work: DEVICE,
 * cs_fit_workspace_bytes bytes. Synchronising. CS_ERR_NUMERIC if the system is not
 * positive definite. */
cs_status cs_fit_workspace_bytes(const cs_ctx* ctx, int n_atoms, int n_basis, size_t* bytes);
cs_status cs_fit_atom_density(cs_ctx* ctx, int n_atoms, const double* atoms, int n_basis,
                              const double* sigmas, const double* target, double ridge,
                              double* coef, void* work, cs_stream stream);

/* The network: n_layers dense layers of sizes dims[0] -> dims[1] -> ... -> dims[n_layers], tanh
 * after every layer but the last. params: HOST initial parameters (FP32, layout above). The
 * network owns its device parameters, Adam moments and scratch for up to max_rows rows. */
typedef struct cs_mlp cs_mlp;
cs_status cs_mlp_create(int n_layers, const int* dims, const float* params, int max_rows,
                        int cuda_device, cs_mlp** out);
cs_status cs_mlp_free(cs_mlp* m);
/* number of parameters (FP32 values) */
cs_status cs_mlp_param_count(const cs_mlp* m, long long* count);
/* HOST copy of the parameters (layout above). Synchronising. */
cs_status cs_mlp_params(const cs_mlp* m, float* params);
/* Y (DEVICE n x dims[n_layers]) = network(X) (DEVICE n x dims[0]); n <= max_rows. */
cs_status cs_mlp_forward(cs_mlp* m, int n, const float* X, float* Y, cs_stream stream);
/* Mean squared error of network(X) against T (DEVICE n x dims[n_layers]) into *loss, and its
 * gradient with respect to every parameter into grads (HOST, or NULL). Synchronising. */
cs_status cs_mlp_loss_grad(cs_mlp* m, int n, const float* X, const float* T, float* loss,
                           float* grads, cs_stream stream);
/* One Adam step (lr; b1 = 0.9, b2 = 0.999, eps = 1e-8, bias-corrected) on the gradient of the
 * mean squared error; *loss receives the loss before the step (if not NULL). Synchronising
 * when loss is not NULL. */
cs_status cs_mlp_train_step(cs_mlp* m, int n, const float* X, const float* T, float lr,
                            float* loss, cs_stream stream);
const char* cs_mlp_last_error(const cs_mlp* m);

#ifdef __cplusplus
}
#endif

#endif /* CLUSTERSPEC_CS_LEARNED_H */
