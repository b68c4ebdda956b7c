"""Pins of the LOBPCG oracle (oracle/lobpcg.py): the Teter-Payne-Allan preconditioner's
limits, convergence to the dense eigenvalues with and without it (and fewer iterations
with it), the free-particle levels, the restart path, and a planted mistake."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import eigen, lobpcg
from oracle.basis import Basis, basis_for
from oracle.hamiltonian import Hamiltonian


def test_tpa_limits():
    """T(g) = 1 - 16 g^4/27 + O(g^5) near 0 (no change to low-energy components, zero
    derivatives up to third order) and T(g) -> 1/(2g) for large g (inverse Laplacian).
    The residual column has its whole weight on the first component, so its kinetic energy
    per unit norm is Lambda_0 / 2 and g = 2 Lambda / Lambda_0."""
    Lam = np.array([1.0, 1e-3, 1e-2, 1e3, 1e6])
    y = np.array([[1.0], [0.0], [0.0], [0.0], [0.0]])
    T = lobpcg.tpa_factors(Lam, y)[:, 0]
    g = 2.0 * Lam
    for gi, ti in zip(g[1:3], T[1:3]):
        assert abs(ti - (1.0 - 16.0 * gi ** 4 / 27.0)) <= gi ** 5
    assert abs(T[4] * 2 * g[4] - 1.0) <= 1e-6
    assert np.all(np.diff(T[[1, 2, 0, 3, 4]]) < 0)  # monotone damping in g


def _small():
    w = W.small_cluster(lmax=5, nmax=8, n_r=16, n_theta=12, n_phi=24, n_s=12, seed=7301)
    b = basis_for(w)
    return w, b, Hamiltonian(b, w.potential_at(b.points()))


@pytest.mark.parametrize("pre", [True, False])
def test_lobpcg_matches_dense(pre):
    w, b, H = _small()
    lam = np.linalg.eigvalsh(H.dense())
    X0 = W.gaussian_block(7302, b.d, 12)
    th, X, res, it, rs = lobpcg.lobpcg(H.apply, X0, 10, 2 * b.half_lambda if pre else None,
                                      tol=1e-9, max_iter=300)
    assert np.max(res[:10]) <= 1e-9
    assert np.max(np.abs(th[:10] - lam[:10])) <= 1e-10
    assert np.max(np.abs(X.T @ X - np.eye(12))) <= 1e-12


def test_tpa_preconditioner_reduces_iterations():
    w, b, H = _small()
    X0 = W.gaussian_block(7303, b.d, 12)
    it_pre = lobpcg.lobpcg(H.apply, X0, 10, 2 * b.half_lambda, tol=1e-8, max_iter=400)[3]
    it_none = lobpcg.lobpcg(H.apply, X0, 10, None, tol=1e-8, max_iter=400)[3]
    assert it_pre < it_none


def test_lobpcg_free_particle_levels():
    """V = 0: the levels 1/2 (z_ln/R)^2, each l level (2l+1)-fold."""
    b = Basis(6.0, 3, 4, 12, 8, 16)
    H = Hamiltonian(b, np.zeros((b.n_r, b.n_theta, b.n_phi)))
    th = lobpcg.lobpcg(H.apply, W.gaussian_block(7304, b.d, 14), 12, 2 * b.half_lambda,
                       tol=1e-10, max_iter=300)[0]
    ref = np.sort(b.half_lambda)[:12]
    assert np.max(np.abs(th[:12] - ref)) <= 1e-10


def test_lobpcg_restart_path():
    """A block with a repeated column breaks the first Cholesky factor of W; the iteration
    restarts from the Ritz vectors and still converges."""
    w, b, H = _small()
    X0 = W.gaussian_block(7305, b.d, 12)
    X0[:, 11] = X0[:, 10] + 1e-14 * X0[:, 9]
    lam = np.linalg.eigvalsh(H.dense())
    th, X, res, it, rs = lobpcg.lobpcg(H.apply, X0, 8, 2 * b.half_lambda, tol=1e-9, max_iter=300)
    assert np.max(np.abs(th[:8] - lam[:8])) <= 1e-9


def test_planted_ignored_overlap_breaks_ritz_values():
    """Planted: the Rayleigh-Ritz step treats S = [X, W, P] as orthonormal (M = I); the Ritz
    values then miss the dense eigenvalues."""
    w, b, H = _small()
    lam = np.linalg.eigvalsh(H.dense())
    X = eigen.cholqr(W.gaussian_block(7306, b.d, 12))
    HX = H.apply(X)
    th, C = np.linalg.eigh(0.5 * (X.T @ HX + HX.T @ X))
    X, HX = X @ C, HX @ C
    with np.errstate(all="ignore"):
        th = _planted_iterations(H, b, X, HX, th)
    # the dense-eigenvalue pin fails (a divergence to non-finite values fails it as well)
    assert not np.allclose(th[:10], lam[:10], atol=1e-3)


def _planted_iterations(H, b, X, HX, th):
    for _ in range(30):
        R = HX - X * th
        Wb = lobpcg.tpa_apply(2 * b.half_lambda, R)  # not orthonormalised
        S = np.concatenate([X, Wb], axis=1)
        HS = np.concatenate([HX, H.apply(Wb)], axis=1)
        Gs = 0.5 * (S.T @ HS + HS.T @ S)
        if not np.all(np.isfinite(Gs)):
            return np.full(12, np.nan)
        t, Q = np.linalg.eigh(Gs)  # overlap ignored
        X, HX, th = S @ Q[:, :12], HS @ Q[:, :12], t[:12]
    return th
