"""LOBPCG with the Teter-Payne-Allan preconditioner (FP64).

Test infrastructure only (see oracle/__init__.py).

Sec. 3.1 (Diagonalization using LOBPCG): locally optimal block preconditioned conjugate
gradients. Each iteration is a Rayleigh-Ritz step on the span of the current Ritz vectors X,
the preconditioned residuals W and the previous search directions P.
- Soft locking: only columns whose residual is above the tolerance contribute W and P.
- The W and P blocks are orthonormalised by Cholesky factors taken after column scaling
  (Sec. 3.1.1), W first against X.
- A breakdown of a factorisation restarts the iteration from the current Ritz vectors
  (W and P discarded), as the paper describes.

Sec. 3.1.2: the diagonal Teter-Payne-Allan preconditioner. For a residual column y,
    g_alpha = Lambda_alpha / (1/2 sum_a Lambda_a y_a^2 / sum_a y_a^2)
(the ratio of the basis function's Laplacian eigenvalue to the residual's kinetic energy per
unit norm) and
    T_alpha = (27 + 18 g + 12 g^2 + 8 g^3) / (27 + 18 g + 12 g^2 + 8 g^3 + 16 g^4).
"""
from __future__ import annotations

import numpy as np

from .eigen import CholeskyBreakdown, cholqr


def tpa_factors(Lam: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Preconditioner diagonal for each column of Y (d, k): T[alpha, s] (Sec. 3.1.2)."""
    Y = np.asarray(Y, dtype=np.float64)
    ke = 0.5 * np.sum(Lam[:, None] * Y * Y, axis=0) / np.sum(Y * Y, axis=0)
    g = Lam[:, None] / ke[None, :]
    num = 27.0 + g * (18.0 + g * (12.0 + 8.0 * g))
    return num / (num + 16.0 * g ** 4)


def tpa_apply(Lam: np.ndarray, Y: np.ndarray) -> np.ndarray:
    return tpa_factors(Lam, Y) * np.asarray(Y, dtype=np.float64)


def _ortho_against(X: np.ndarray, W: np.ndarray) -> np.ndarray:
    return W - X @ (X.T @ W)


def lobpcg(apply_H, X0: np.ndarray, n_want: int, Lam: np.ndarray | None = None,
           tol: float = 1e-8, max_iter: int = 200):
    """Lowest n_s = X0.shape[1] eigenpairs of the symmetric operator apply_H. Convergence:
    the largest residual ||H x_i - theta_i x_i|| over the n_want lowest pairs <= tol.
    Lam: Laplacian eigenvalue of each basis function (TPA preconditioner), or None (no
    preconditioner). Returns (theta, X, residual norms, iterations, restarts)."""
    X = cholqr(np.asarray(X0, dtype=np.float64))
    HX = apply_H(X)
    th, C = np.linalg.eigh(0.5 * (X.T @ HX + HX.T @ X))
    X, HX = X @ C, HX @ C
    m = X.shape[1]
    P = HP = None
    restarts = 0
    res = None
    for it in range(1, max_iter + 1):
        R = HX - X * th[None, :]
        res = np.linalg.norm(R, axis=0)
        if np.max(res[:n_want]) <= tol:
            return th, X, res, it - 1, restarts
        act = np.nonzero(res > tol)[0]
        W = R[:, act]
        if Lam is not None:
            W = tpa_apply(Lam, W)
        try:
            W = cholqr(_ortho_against(X, W))
            HW = apply_H(W)
            blocks, hblocks = [X, W], [HX, HW]
            if P is not None:
                Pa, HPa = P[:, act], HP[:, act]
                # orthonormalise P_a by the Cholesky factor of its Gram (the same U applied
                # to H P_a), after column scaling
                U = _chol_factor(Pa.T @ Pa)
                blocks.append(Pa @ U)
                hblocks.append(HPa @ U)
            S = np.concatenate(blocks, axis=1)
            HS = np.concatenate(hblocks, axis=1)
            G = 0.5 * (S.T @ HS + HS.T @ S)
            U = _chol_factor(S.T @ S)  # U^T M U = I
            t, Q = np.linalg.eigh(0.5 * (U.T @ G @ U + (U.T @ G @ U).T))
            Cm = U @ Q[:, :m]
        except CholeskyBreakdown:
            P = HP = None
            restarts += 1
            continue
        X, HX = S @ Cm, HS @ Cm
        P, HP = S[:, m:] @ Cm[m:, :], HS[:, m:] @ Cm[m:, :]
        th = t[:m]
    R = HX - X * th[None, :]
    return th, X, np.linalg.norm(R, axis=0), max_iter, restarts


def _chol_factor(M: np.ndarray) -> np.ndarray:
    """U = D R^{-1} with D = diag(M)^(-1/2) and D M D = R^T R, so that U^T M U = I
    (Cholesky after column scaling, Sec. 3.1.1)."""
    dg = np.diag(M)
    if np.any(dg <= 0.0) or not np.all(np.isfinite(dg)):
        raise CholeskyBreakdown("zero or non-finite diagonal")
    D = 1.0 / np.sqrt(dg)
    try:
        L = np.linalg.cholesky(D[:, None] * M * D[None, :])
    except np.linalg.LinAlgError as e:
        raise CholeskyBreakdown(str(e)) from e
    return D[:, None] * np.linalg.inv(L.T)
