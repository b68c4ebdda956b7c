"""Learned initial SCF density (FP64): per-atom radial descriptors, atom-centred radial density
corrections fitted to converged densities, a small multilayer perceptron that maps the one to
the other, and the density it predicts.

Test infrastructure only (see oracle/__init__.py).

The method's SCF needs a starting density (Sec. 3.2.1 uses the superposition of atomic
densities). This form learns a correction to that start.
- **Descriptor** of atom a: D_ak = sum_{b != a} exp(-(r_ab - mu_k)^2 / (2 w^2)), neighbour
  counts in soft radial shells. It is invariant under rotations, translations and permutations
  of the other atoms.
- **Radial basis**: phi_j(r) = (2 pi s_j^2)^(-3/2) exp(-r^2 / (2 s_j^2)), unit-integral
  Gaussians of widths s_j.
- **Correction**: drho(x) = sum_a sum_j c_aj phi_j(|x - a|).
- **Targets**: the coefficients c that best fit rho_converged - rho_start on the grid in the
  quadrature-weighted least-squares sense (normal equations with a small ridge term).
- **Network**: an MLP D -> tanh(W1 . + b1) -> ... -> W_L . + b_L (linear output), trained on
  the mean squared error over atoms and outputs with Adam (Kingma & Ba 2015, the published
  update with bias correction).
- **Prediction**: rho0 = rho_start + drho, rescaled to integrate to the electron count.
"""
from __future__ import annotations

import math

import numpy as np


def descriptors(atoms: np.ndarray, mu: np.ndarray, width: float) -> np.ndarray:
    atoms = np.asarray(atoms, dtype=np.float64)
    n = atoms.shape[0]
    r = np.linalg.norm(atoms[:, None, :] - atoms[None, :, :], axis=2)
    g = np.exp(-((r[:, :, None] - mu[None, None, :]) ** 2) / (2.0 * width * width))
    g[np.arange(n), np.arange(n), :] = 0.0
    return g.sum(axis=1)


def radial_basis(r: np.ndarray, sigmas: np.ndarray) -> np.ndarray:
    """phi_j(r) for each point (rows) and width (columns)."""
    s = np.asarray(sigmas, dtype=np.float64)[None, :]
    return (2.0 * math.pi * s * s) ** -1.5 * np.exp(-(np.asarray(r)[:, None] ** 2) / (2.0 * s * s))


def correction(points: np.ndarray, atoms: np.ndarray, sigmas: np.ndarray,
               coef: np.ndarray) -> np.ndarray:
    """drho at the points: sum_a sum_j coef[a, j] phi_j(|x - a|)."""
    out = np.zeros(points.shape[0])
    for a, c in zip(np.asarray(atoms), np.asarray(coef)):
        out += radial_basis(np.linalg.norm(points - a[None, :], axis=1), sigmas) @ c
    return out


def fit_coefficients(points: np.ndarray, weights: np.ndarray, atoms: np.ndarray,
                     sigmas: np.ndarray, target: np.ndarray, ridge: float = 1e-10) -> np.ndarray:
    """argmin_c sum_g W_g (sum_{a,j} c_aj phi_j(|x_g - a|) - target_g)^2 + ridge |c|^2, by the
    normal equations (M + ridge tr(M)/n I) c = A^T W target with M = A^T W A."""
    cols = []
    for a in np.asarray(atoms):
        cols.append(radial_basis(np.linalg.norm(points - a[None, :], axis=1), sigmas))
    A = np.concatenate(cols, axis=1)
    w = np.asarray(weights, dtype=np.float64).ravel()
    M = A.T @ (w[:, None] * A)
    rhs = A.T @ (w * np.asarray(target, dtype=np.float64).ravel())
    M = M + ridge * np.trace(M) / M.shape[0] * np.eye(M.shape[0])
    c = np.linalg.solve(M, rhs)
    return c.reshape(len(atoms), len(sigmas))


class MLP:
    """Fully connected network with tanh hidden layers and a linear output."""

    def __init__(self, params: list):
        # params: [W1, b1, W2, b2, ...], W_i shape (n_in, n_out)
        self.params = [np.array(p, dtype=np.float64) for p in params]

    @property
    def n_layers(self) -> int:
        return len(self.params) // 2

    def forward(self, X: np.ndarray, keep: bool = False):
        acts = [np.asarray(X, dtype=np.float64)]
        h = acts[0]
        for i in range(self.n_layers):
            W, b = self.params[2 * i], self.params[2 * i + 1]
            z = h @ W + b[None, :]
            h = np.tanh(z) if i < self.n_layers - 1 else z
            acts.append(h)
        return (h, acts) if keep else h

    def loss_and_grads(self, X: np.ndarray, T: np.ndarray):
        """Mean squared error L = mean over all entries of (Y - T)^2 and its gradients."""
        Y, acts = self.forward(X, keep=True)
        diff = Y - T
        n = diff.size
        loss = float(np.sum(diff * diff) / n)
        grads = [None] * len(self.params)
        d = 2.0 * diff / n  # dL/dY
        for i in reversed(range(self.n_layers)):
            W = self.params[2 * i]
            h_in = acts[i]
            if i < self.n_layers - 1:
                d = d * (1.0 - acts[i + 1] ** 2)  # through tanh
            grads[2 * i] = h_in.T @ d
            grads[2 * i + 1] = d.sum(axis=0)
            d = d @ W.T
        return loss, grads


class Adam:
    """Adam with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, params: list, lr: float, b1: float = 0.9, b2: float = 0.999,
                 eps: float = 1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0

    def step(self, params: list, grads: list):
        self.t += 1
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.b1
            m += (1.0 - self.b1) * g
            v *= self.b2
            v += (1.0 - self.b2) * g * g
            mh = m / (1.0 - self.b1 ** self.t)
            vh = v / (1.0 - self.b2 ** self.t)
            p -= self.lr * mh / (np.sqrt(vh) + self.eps)


def predicted_density(points, weights, atoms, sigmas, coef, rho_start, n_electrons):
    """rho0 = rho_start + drho, scaled to integrate to n_electrons."""
    rho = np.asarray(rho_start, dtype=np.float64).ravel() + correction(points, atoms, sigmas, coef)
    return rho * (n_electrons / float(np.sum(np.asarray(weights).ravel() * rho)))
