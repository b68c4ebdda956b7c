"""Spherical spectral basis, quadrature grid and basis transforms (FP64).

Test infrastructure only (see oracle/__init__.py).

Basis (Sec. 2.2.1): F_lmn(r, theta, phi) = R_ln(r) Y_lm(theta, phi) on the ball of
radius R, 0 <= l < L, -l <= m <= l, 0 <= n < N, so d = L^2 N.
  R_ln(r) = sqrt(2/R^3) j_l(z_ln r / R) / j_{l+1}(z_ln)      (eq. spherical_bessel_1,
            rewritten with j_l(x) = sqrt(pi/(2x)) J_{l+1/2}(x); the sign of the
            denominator is kept as printed)
  Lambda_ln = (z_ln / R)^2                                    (eq. laplacian_eigenvalue)
Real harmonics (the real-function symmetry of Sec. 2.2.1 maps the complex Y_l^{+-m} onto
these one to one; no Condon-Shortley phase):
  Y_l0 = Theta_l0(cos theta),  Y_lm = sqrt2 Theta_lm cos(m phi),
  Y_l,-m = sqrt2 Theta_lm sin(m phi)   (m > 0)
Index map (footnote to eq. Hij_def, 0-based): alpha(l, m, n) = (l^2 + l + m) N + n.

Grid (Sec. 2.2.2): N_r radial nodes on [0, R] with weights that include r^2 (Gauss-
Jacobi for the weight r^2, or Gauss-Legendre with r^2 folded into the weights),
N_theta Gauss points in t = cos(theta) (ascending t), N_phi uniform points
phi_q = 2 pi q / N_phi with weight 2 pi / N_phi. Grid functions are arrays [k][j][q].
"""
from __future__ import annotations

import math

import numpy as np

from .special import (gauss_jacobi_0_2, gauss_legendre, norm_assoc_legendre, sph_bessel_j,
                      sph_bessel_zeros)


def alpha(l: int, m: int, n: int, N: int) -> int:
    """0-based index of basis function (l, m, n)."""
    return (l * l + l + m) * N + n


class Basis:
    """Tables of the basis on its quadrature grid.

    radial[l]  : (N_r, N)      R_ln(r_k)
    theta[m]   : (N_theta, L-m) Theta_lm(t_j) for l = m .. lmax
    phi_fn     : (N_phi, 2L-1) column m + lmax holds 1, sqrt2 cos(m phi_q) (m > 0) or
                 sqrt2 sin(|m| phi_q) (m < 0)
    half_lambda: (d,)          1/2 Lambda_{l,n} at alpha(l, m, n)
    """

    def __init__(self, R: float, lmax: int, nmax: int, n_r: int, n_theta: int, n_phi: int,
                 radial_rule: str = "gauss_legendre"):
        self.R = float(R)
        self.lmax = int(lmax)
        self.L = self.lmax + 1
        self.N = int(nmax)
        self.d = self.L * self.L * self.N
        self.n_r, self.n_theta, self.n_phi = int(n_r), int(n_theta), int(n_phi)
        self.radial_rule = radial_rule
        L, N = self.L, self.N

        # radial nodes and weights (weights include r^2), Sec. 2.2.2
        if radial_rule == "gauss_legendre":
            x, w = gauss_legendre(self.n_r)
            self.r = 0.5 * self.R * (1.0 + x)
            self.w_r = 0.5 * self.R * w * self.r ** 2
        elif radial_rule == "gauss_jacobi_r2":
            x, w = gauss_jacobi_0_2(self.n_r)
            self.r = 0.5 * self.R * (1.0 + x)
            self.w_r = (0.5 * self.R) ** 3 * w
        else:
            raise ValueError(radial_rule)
        self.t, self.w_t = gauss_legendre(self.n_theta)
        self.phi = 2.0 * np.pi * np.arange(self.n_phi) / self.n_phi
        self.w_phi = 2.0 * np.pi / self.n_phi

        # Bessel zeros and radial functions, eqs. spherical_bessel_1, laplacian_eigenvalue
        self.z = sph_bessel_zeros(self.lmax, self.N)
        self.radial = []
        for l in range(L):
            k = self.z[l] / self.R
            norm = math.sqrt(2.0 / self.R ** 3) / np.array(
                [sph_bessel_j(l + 1, self.z[l, n])[0] for n in range(N)])
            tab = np.empty((self.n_r, N))
            for n in range(N):
                tab[:, n] = norm[n] * sph_bessel_j(l, k[n] * self.r)
            self.radial.append(tab)

        # normalised associated Legendre functions, eq. spherical_harmonics_1
        th = norm_assoc_legendre(self.lmax, self.t)
        self.theta = [th[m:, m, :].T.copy() for m in range(L)]

        # phi functions of the real harmonics
        self.phi_fn = np.empty((self.n_phi, 2 * L - 1))
        for m in range(-self.lmax, L):
            if m == 0:
                self.phi_fn[:, m + self.lmax] = 1.0
            elif m > 0:
                self.phi_fn[:, m + self.lmax] = math.sqrt(2.0) * np.cos(m * self.phi)
            else:
                self.phi_fn[:, m + self.lmax] = math.sqrt(2.0) * np.sin(-m * self.phi)

        hl = np.empty(self.d)
        for l in range(L):
            for m in range(-l, l + 1):
                a0 = alpha(l, m, 0, N)
                hl[a0:a0 + N] = 0.5 * (self.z[l] / self.R) ** 2
        self.half_lambda = hl

    # ------------------------------------------------------------------ grid helpers
    @property
    def n_grid(self) -> int:
        return self.n_r * self.n_theta * self.n_phi

    def points(self) -> np.ndarray:
        """Cartesian coordinates of the grid, (N_g, 3), order [k][j][q]."""
        st = np.sqrt(1.0 - self.t ** 2)
        r = self.r[:, None, None]
        x = r * st[None, :, None] * np.cos(self.phi)[None, None, :]
        y = r * st[None, :, None] * np.sin(self.phi)[None, None, :]
        zz = r * self.t[None, :, None] * np.ones(self.n_phi)[None, None, :]
        return np.stack([x.ravel(), y.ravel(), zz.ravel()], axis=1)

    def weights(self) -> np.ndarray:
        """Quadrature weights W[k, j, q] = w_r[k] w_t[j] 2pi/N_phi."""
        return (self.w_r[:, None, None] * self.w_t[None, :, None]
                * np.full(self.n_phi, self.w_phi)[None, None, :])

    # ------------------------------------------------------------------ transforms
    def inverse_transform(self, X: np.ndarray) -> np.ndarray:
        """Coefficients X (d, S) -> grid values f (N_r, N_theta, N_phi, S).

        Step 1 (eq. G_lmr): G_l[k, m, s] = sum_n R_ln(r_k) X[alpha(l,m,n), s].
        Step 2 (inverse spherical harmonic transform at each radial node, Sec. 2.2.2):
          Legendre sums  F_m[k, j, s] = sum_{l >= |m|} Theta_l|m|(t_j) G_l[k, m, s],
          phi sums       f[k, j, q, s] = sum_m phi_fn[q, m] F_m[k, j, s].
        """
        L, N, lmax = self.L, self.N, self.lmax
        S = X.shape[1]
        G = []
        for l in range(L):
            Xl = X[l * l * N:(l + 1) * (l + 1) * N, :].reshape(2 * l + 1, N, S)
            G.append(np.einsum("kn,mns->kms", self.radial[l], Xl))
        F = np.empty((2 * L - 1, self.n_r, self.n_theta, S))
        for m in range(-lmax, L):
            am = abs(m)
            Gm = np.stack([G[l][:, l + m, :] for l in range(am, L)], axis=0)  # (L-|m|, N_r, S)
            F[m + lmax] = np.einsum("jl,lks->kjs", self.theta[am], Gm)
        return np.einsum("qm,mkjs->kjqs", self.phi_fn, F)

    def forward_transform(self, g: np.ndarray) -> np.ndarray:
        """Grid values g (N_r, N_theta, N_phi, S) -> coefficients (d, S) by quadrature.

        eq. Ar_lm: A(r_k; l, m) = sum_j w_t[j] Theta_l|m|(t_j)
                                  [sum_q (2 pi/N_phi) phi_fn[q, m] g[k, j, q]],
        eq. Arlm_to_coeff: coeff(l, m, n) = sum_k w_r[k] A(r_k; l, m) R_ln(r_k).
        """
        L, N, lmax = self.L, self.N, self.lmax
        S = g.shape[3]
        A = self.w_phi * np.einsum("qm,kjqs->mkjs", self.phi_fn, g)  # (2L-1, N_r, N_th, S)
        out = np.empty((self.d, S))
        for l in range(L):
            Al = np.empty((self.n_r, 2 * l + 1, S))
            for m in range(-l, l + 1):
                am = abs(m)
                coef = self.w_t * self.theta[am][:, l - am]
                Al[:, m + l, :] = np.einsum("j,kjs->ks", coef, A[m + lmax])
            Zl = np.einsum("k,kn,kms->mns", self.w_r, self.radial[l], Al)
            out[l * l * N:(l + 1) * (l + 1) * N, :] = Zl.reshape((2 * l + 1) * N, S)
        return out

    # ------------------------------------------------------------------ explicit matrix
    def synthesis_matrix(self) -> np.ndarray:
        """B[g, alpha] = F_alpha(x_g) for tiny bases (N_g x d, explicit)."""
        L, N, lmax = self.L, self.N, self.lmax
        B = np.empty((self.n_r, self.n_theta, self.n_phi, self.d))
        for l in range(L):
            for m in range(-l, l + 1):
                am = abs(m)
                ang = self.theta[am][:, l - am][:, None] * self.phi_fn[:, m + lmax][None, :]
                for n in range(N):
                    B[:, :, :, alpha(l, m, n, N)] = (self.radial[l][:, n][:, None, None]
                                                      * ang[None, :, :])
        return B.reshape(self.n_grid, self.d)


def basis_for(w) -> Basis:
    """Basis of a workload description (workloads.Workload)."""
    return Basis(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, w.radial_rule)
