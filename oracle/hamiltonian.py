"""Matrix-free Hamiltonian product and its explicit dense form (FP64).

Test infrastructure only (see oracle/__init__.py).

Sec. 2.2.4, eq. matvec_final: Z = 1/2 Lambda . Y + <V_eff (sum_b Y_b F_b), F_a>, computed as
kinetic part in coefficient space plus an inverse basis transform, a pointwise product
with V_eff on the grid and a forward basis transform. The inner product is the grid
quadrature, so the operator applied is

    H = 1/2 diag(Lambda) + B^T diag(W V) B + P diag(h) P^T

with B the synthesis matrix and W the quadrature weights. The last term is the non-local
Kleinman-Bylander part (Sec. 2.3.2): projector functions are sampled on the grid and
forward transformed once; their action on a block is a pair of matrix products.
"""
from __future__ import annotations

import numpy as np

from .basis import Basis


class Hamiltonian:
    """H for a fixed basis, effective potential on the grid and optional projectors."""

    def __init__(self, basis: Basis, v_grid: np.ndarray, proj_grid: np.ndarray | None = None,
                 h: np.ndarray | None = None):
        self.basis = basis
        self.v = np.asarray(v_grid, dtype=np.float64).reshape(basis.n_r, basis.n_theta,
                                                               basis.n_phi)
        self.P = None
        self.h = None
        if proj_grid is not None:
            pg = np.asarray(proj_grid, dtype=np.float64).reshape(-1, basis.n_r, basis.n_theta,
                                                                 basis.n_phi)
            # coefficients of each projector by forward transform (Sec. 2.3.2)
            self.P = basis.forward_transform(np.moveaxis(pg, 0, -1))  # (d, N_p)
            self.h = np.asarray(h, dtype=np.float64)

    def apply(self, X: np.ndarray, chunk: int = 64) -> np.ndarray:
        """H X for a block X (d, S): kinetic + transform sandwich + projector pair."""
        X = np.asarray(X, dtype=np.float64)
        if X.ndim == 1:
            return self.apply(X[:, None], chunk)[:, 0]
        b = self.basis
        out = np.empty_like(X)
        for s0 in range(0, X.shape[1], chunk):
            Xc = X[:, s0:s0 + chunk]
            f = b.inverse_transform(Xc)                   # real-space states
            g = self.v[:, :, :, None] * f                 # pointwise V_eff
            out[:, s0:s0 + chunk] = b.half_lambda[:, None] * Xc + b.forward_transform(g)
        if self.P is not None:
            out += self.P @ (self.h[:, None] * (self.P.T @ X))
        return out

    def dense(self) -> np.ndarray:
        """Explicit H = 1/2 diag(Lambda) + B^T diag(W V) B + P diag(h) P^T (tiny bases)."""
        b = self.basis
        B = b.synthesis_matrix()
        wv = (b.weights() * self.v).ravel()
        H = B.T @ (wv[:, None] * B)
        H[np.diag_indices_from(H)] += b.half_lambda
        if self.P is not None:
            H += self.P @ (self.h[:, None] * self.P.T)
        return H
