"""Chebyshev-filtered subspace iteration and its pieces (FP64).

Test infrastructure only (see oracle/__init__.py).

Sec. 3.2 / 3.2.1: each iteration filters the block with a Chebyshev polynomial in H
(built from H.X products and scale/shift operations), orthonormalises it by a Cholesky
factorisation (in place of DGKS), and performs a Rayleigh-Ritz step. Sec. 3.1.1: Cholesky
factors are taken after column scaling. The filter is the scaled three-term form of the
method the paper cites (Zhou, Saad et al.); the bounds come from a short Lanczos run.

    c = (a+b)/2, e = (b-a)/2, sigma_1 = e/(a0 - c), Y_0 = X,
    Y_1 = (sigma_1/e)(H - c) X,
    sigma_{i+1} = 1/(2/sigma_1 - sigma_i),
    Y_{i+1} = (2 sigma_{i+1}/e)(H - c) Y_i - sigma_i sigma_{i+1} Y_{i-1},
    result Y_m = T_m((H - c)/e) X / T_m((a0 - c)/e).
"""
from __future__ import annotations

import numpy as np


def chebyshev_sigmas(m: int, a: float, b: float, a0: float) -> np.ndarray:
    """sigma_1 .. sigma_m of the scaled recurrence (index 0 holds sigma_1)."""
    c = 0.5 * (a + b)
    e = 0.5 * (b - a)
    s = np.empty(m)
    s[0] = e / (a0 - c)
    for i in range(1, m):
        s[i] = 1.0 / (2.0 / s[0] - s[i - 1])
    return s


def cheb_filter(apply_H, X: np.ndarray, m: int, a: float, b: float, a0: float) -> np.ndarray:
    """Y_m = p_m(H) X by the scaled three-term recurrence (degree m >= 1)."""
    c = 0.5 * (a + b)
    e = 0.5 * (b - a)
    sig = chebyshev_sigmas(m, a, b, a0)
    Y_prev = np.array(X, dtype=np.float64, copy=True)
    Y = (sig[0] / e) * (apply_H(Y_prev) - c * Y_prev)
    for i in range(1, m):
        s_new = sig[i]
        Y_new = (2.0 * s_new / e) * (apply_H(Y) - c * Y) - (sig[i - 1] * s_new) * Y_prev
        Y_prev, Y = Y, Y_new
    return Y


class CholeskyBreakdown(RuntimeError):
    pass


def cholqr(X: np.ndarray, passes: int = 2) -> np.ndarray:
    """Orthonormalise the columns of X: M = X^T X, D = diag(M)^(-1/2),
    D M D = R^T R (Cholesky, R upper), X <- X D R^{-1}; repeated `passes` times."""
    X = np.array(X, dtype=np.float64, copy=True)
    for _ in range(passes):
        M = X.T @ X
        dg = np.diag(M)
        if np.any(dg <= 0.0) or not np.all(np.isfinite(dg)):
            raise CholeskyBreakdown("zero or non-finite column")
        D = 1.0 / np.sqrt(dg)
        Ms = D[:, None] * M * D[None, :]
        try:
            Lc = np.linalg.cholesky(Ms)  # Ms = Lc Lc^T, R = Lc^T
        except np.linalg.LinAlgError as exc:
            raise CholeskyBreakdown(str(exc)) from exc
        Rinv = np.linalg.inv(Lc.T)
        X = X @ (D[:, None] * Rinv)
    return X


def rayleigh_ritz(apply_H, X: np.ndarray):
    """For orthonormal X: Hs = 1/2 (X^T H X + (X^T H X)^T) = Q Theta Q^T,
    X <- X Q, HX <- (H X) Q, residuals rho_i = ||HX_i - theta_i X_i||_2."""
    HX = apply_H(X)
    Hs = X.T @ HX
    Hs = 0.5 * (Hs + Hs.T)
    theta, Q = np.linalg.eigh(Hs)
    Xr = X @ Q
    HXr = HX @ Q
    resid = np.linalg.norm(HXr - Xr * theta[None, :], axis=0)
    return theta, Xr, HXr, resid


def lanczos_bound(apply_H, v0: np.ndarray, k: int = 10):
    """k-step Lanczos (full reorthogonalisation) from v0.

    Returns (b, theta_min): b = largest Ritz value + |beta_k| (an upper bound of the
    spectrum used by the filter), theta_min = smallest Ritz value.
    """
    d = v0.size
    k = min(k, d)
    V = np.zeros((d, k))
    alphas = np.zeros(k)
    betas = np.zeros(k)
    v = v0 / np.linalg.norm(v0)
    for i in range(k):
        V[:, i] = v
        w = apply_H(v)
        alphas[i] = v @ w
        w = w - V[:, :i + 1] @ (V[:, :i + 1].T @ w)
        w = w - V[:, :i + 1] @ (V[:, :i + 1].T @ w)
        betas[i] = np.linalg.norm(w)
        if betas[i] == 0.0:
            k = i + 1
            break
        v = w / betas[i]
    T = np.diag(alphas[:k]) + np.diag(betas[:k - 1], 1) + np.diag(betas[:k - 1], -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] + abs(betas[k - 1])), float(ev[0])


def chfsi(apply_H, X0: np.ndarray, n_want: int, degree: int, v0: np.ndarray,
          tol: float = 1e-8, max_iter: int = 50, lanczos_steps: int = 10):
    """ChFSI from a given block: bounds, then [filter -> CholQR -> Rayleigh-Ritz]
    until the largest residual among the n_want lowest Ritz pairs is <= tol.

    First pass: a0 = smallest Lanczos Ritz value, a = a0 + (b - a0)/10; later passes:
    a = largest Ritz value of the block, a0 = smallest.
    Returns (theta, X, resid, iterations).
    """
    b, tmin = lanczos_bound(apply_H, v0, lanczos_steps)
    a0 = tmin
    a = a0 + (b - a0) / 10.0
    X = cholqr(X0)
    theta = resid = None
    it = 0
    for it in range(1, max_iter + 1):
        Y = cheb_filter(apply_H, X, degree, a, b, a0)
        X = cholqr(Y)
        theta, X, _, resid = rayleigh_ritz(apply_H, X)
        if np.max(resid[:n_want]) <= tol:
            break
        a = float(theta[-1])
        a0 = float(theta[0])
    return theta, X, resid, it
