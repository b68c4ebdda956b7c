"""Pins for oracle/eigen.py: the Chebyshev filter against its closed form through a
dense eigendecomposition, the sigma recurrence against T_i ratios, Cholesky-QR, the
Rayleigh-Ritz step, the Lanczos bound and the ChFSI loop against dense eigenvalues."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen
from oracle.basis import Basis, basis_for
from oracle.hamiltonian import Hamiltonian


def _cheb_T(m, x):
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    inside = np.abs(x) <= 1
    out[inside] = np.cos(m * np.arccos(x[inside]))
    xo = x[~inside]
    out[~inside] = np.sign(xo) ** m * np.cosh(m * np.arccosh(np.abs(xo)))
    return out


def _small():
    w = W.small_cluster()
    b = basis_for(w)
    return w, b, Hamiltonian(b, w.potential_at(b.points()))


def test_sigmas_are_chebyshev_ratios():
    a, b, a0 = 3.0, 50.0, -5.0
    c, e = 0.5 * (a + b), 0.5 * (b - a)
    s = eigen.chebyshev_sigmas(12, a, b, a0)
    T = [_cheb_T(i, np.array([(a0 - c) / e]))[0] for i in range(13)]
    assert np.allclose(s, [T[i] / T[i + 1] for i in range(12)], rtol=1e-13)


@pytest.mark.parametrize("m", [1, 2, 7, 16])
def test_filter_closed_form(m):
    w, b, H = _small()
    Hd = H.dense()
    lam, Q = np.linalg.eigh(Hd)
    a, bb, a0 = float(lam[20]), float(lam[-1]) + 0.5, float(lam[0])
    c, e = 0.5 * (a + bb), 0.5 * (bb - a)
    X = W.gaussian_block(77, b.d, 5)
    got = eigen.cheb_filter(H.apply, X, m, a, bb, a0)
    gain = _cheb_T(m, (lam - c) / e) / _cheb_T(m, np.array([(a0 - c) / e]))[0]
    ref = Q @ (gain[:, None] * (Q.T @ X))
    assert np.max(np.abs(got - ref)) < 1e-11 * np.abs(ref).max()


def test_filter_with_zero_potential_is_elementwise():
    b = Basis(5.0, 3, 5, 12, 8, 16)
    H = Hamiltonian(b, np.zeros(b.n_grid))
    lam = b.half_lambda
    a, bb, a0 = 30.0, float(lam.max()) + 1.0, float(lam.min())
    c, e = 0.5 * (a + bb), 0.5 * (bb - a)
    X = W.gaussian_block(3, b.d, 2)
    got = eigen.cheb_filter(H.apply, X, 9, a, bb, a0)
    gain = _cheb_T(9, (lam - c) / e) / _cheb_T(9, np.array([(a0 - c) / e]))[0]
    assert np.allclose(got, gain[:, None] * X, rtol=1e-12, atol=1e-14 * np.abs(got).max())


def test_cholqr_orthonormal_and_same_span():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((300, 12)) @ np.diag(np.logspace(0, 6, 12))
    Q = eigen.cholqr(X)
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) < 1e-14
    # Q = X U for upper-triangular U: the leading k columns span the same spaces
    U = np.linalg.lstsq(X, Q, rcond=None)[0]
    assert np.max(np.abs(np.tril(U, -1))) < 1e-10 * np.abs(U).max()
    assert np.max(np.abs(X @ U - Q)) < 1e-10  # lstsq on columns scaled up to 1e6


def test_cholqr_breakdown_raises():
    X = np.ones((50, 3))
    with pytest.raises(eigen.CholeskyBreakdown):
        eigen.cholqr(X)


def test_rayleigh_ritz_exact_on_invariant_subspace():
    w, b, H = _small()
    lam, Q = np.linalg.eigh(H.dense())
    rng = np.random.default_rng(4)
    rot, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    X = Q[:, :6] @ rot
    theta, Xr, HXr, resid = eigen.rayleigh_ritz(H.apply, X)
    assert np.max(np.abs(theta - lam[:6])) < 1e-12
    assert np.max(resid) < 1e-11


def test_lanczos_bound_is_upper_bound():
    w, b, H = _small()
    lam = np.linalg.eigvalsh(H.dense())
    for seed in [1, 2, 3]:
        bnd, tmin = eigen.lanczos_bound(H.apply, W.gaussian(seed, b.d), 10)
        assert bnd >= lam[-1]
        assert tmin >= lam[0] - 1e-12
        assert bnd < 2.0 * lam[-1] + 10.0  # not absurdly loose


def test_chfsi_matches_dense_eigenvalues():
    w, b, H = _small()
    lam = np.linalg.eigvalsh(H.dense())
    n_want = 6
    theta, X, resid, it = eigen.chfsi(H.apply, w.x_block(), n_want, 10, W.gaussian(9, b.d),
                                      tol=1e-10, max_iter=100)
    assert np.max(resid[:n_want]) <= 1e-10
    assert np.max(np.abs(theta[:n_want] - lam[:n_want])) < 1e-12


def test_chfsi_harmonic_oscillator_workload():
    w = W.harmonic_oscillator_ball()
    b = basis_for(w)
    H = Hamiltonian(b, w.potential_at(b.points()))
    theta, X, resid, it = eigen.chfsi(H.apply, w.x_block(), w.n_want, w.degree,
                                      W.gaussian(99, b.d), tol=1e-8, max_iter=60)
    lev = np.array([1.5] + [2.5] * 3 + [3.5] * 6)
    assert np.max(np.abs(theta[:10] - lev)) < 1e-6
    assert np.max(resid[:10]) <= 1e-8


def test_planted_wrong_sigma_sign_breaks_filter_closed_form():
    w, b, H = _small()
    lam, Q = np.linalg.eigh(H.dense())
    a, bb, a0 = float(lam[20]), float(lam[-1]) + 0.5, float(lam[0])
    c, e = 0.5 * (a + bb), 0.5 * (bb - a)
    X = W.gaussian_block(77, b.d, 2)
    # planted: the three-term recurrence with + instead of - on the Y_{i-1} term
    sig = eigen.chebyshev_sigmas(5, a, bb, a0)
    Yp, Y = X, (sig[0] / e) * (H.apply(X) - c * X)
    for i in range(1, 5):
        Yn = (2 * sig[i] / e) * (H.apply(Y) - c * Y) + sig[i - 1] * sig[i] * Yp
        Yp, Y = Y, Yn
    gain = _cheb_T(5, (lam - c) / e) / _cheb_T(5, np.array([(a0 - c) / e]))[0]
    ref = Q @ (gain[:, None] * (Q.T @ X))
    assert np.max(np.abs(Y - ref)) > 1e-3 * np.abs(ref).max()


def test_chfsi_free_particle_levels_and_multiplicities():
    """V = 0: the ChFSI eigenvalues are the free-particle levels 1/2 (z_ln/R)^2, each l level
    (2l+1)-fold degenerate (Sec. 2.2.1), taken from the Bessel zeros in closed form order."""
    from oracle.basis import Basis
    from oracle.hamiltonian import Hamiltonian
    b = Basis(6.0, 3, 6, n_r=20, n_theta=8, n_phi=16)
    H = Hamiltonian(b, np.zeros(b.n_grid))
    levels = sorted(0.5 * (b.z[l, n] / b.R) ** 2 for l in range(b.L) for n in range(b.N)
                    for _ in range(2 * l + 1))
    # ten wanted levels: the next level is the sevenfold l = 3 one, wholly inside the block
    X0 = W.gaussian_block(61, b.d, 17)
    theta, X, resid, it = eigen.chfsi(H.apply, X0, 10, 10, W.gaussian(62, b.d), tol=1e-10)
    assert np.max(np.abs(theta[:10] - np.array(levels[:10]))) < 1e-10
