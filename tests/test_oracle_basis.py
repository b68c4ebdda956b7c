"""Pins for oracle/basis.py: basis functions against closed forms and scipy's spherical
harmonics, discrete orthonormality under the quadrature, transform round trips."""
import math

import numpy as np
import pytest
from scipy import special as sp

from oracle.basis import Basis, alpha
from oracle.special import sph_bessel_j


def test_radial_l0_closed_form():
    # R_0n(r) = (-1)^n sqrt(2/R) sin((n+1) pi r / R) / r
    b = Basis(8.0, 2, 12, 40, 6, 10)
    r = b.r
    for n in range(12):
        ref = (-1) ** n * math.sqrt(2.0 / b.R) * np.sin((n + 1) * math.pi * r / b.R) / r
        assert np.max(np.abs(b.radial[0][:, n] - ref)) < 1e-13


def test_radial_continuous_normalisation():
    # int_0^R R_ln(r)^2 r^2 dr = 1, with a high-order rule (independent of the config grid)
    b = Basis(6.0, 8, 10, 200, 4, 8)
    for l in [0, 3, 8]:
        M = (b.radial[l] * b.w_r[:, None]).T @ b.radial[l]
        assert np.max(np.abs(M - np.eye(10))) < 1e-13


def test_radial_vanishes_at_boundary_and_laplacian_eigenvalue():
    # F_ln satisfies -(1/r^2)(r^2 R')' + l(l+1)/r^2 R = Lambda R, and R(R_ball) = 0
    R = 5.0
    b = Basis(R, 6, 5, 20, 4, 8)
    for l in [0, 2, 6]:
        for n in [0, 3]:
            k = b.z[l, n] / R
            c = math.sqrt(2.0 / R ** 3) / sph_bessel_j(l + 1, b.z[l, n])[0]
            f = lambda r: c * sph_bessel_j(l, k * np.asarray(r))
            assert abs(f(R)[0]) < 1e-14
            r0, h = np.array([1.3, 2.9]), 1e-3
            d1 = (f(r0 + h) - f(r0 - h)) / (2 * h)
            d2 = (f(r0 + h) - 2 * f(r0) + f(r0 - h)) / h ** 2
            lap = d2 + 2 / r0 * d1 - l * (l + 1) / r0 ** 2 * f(r0)
            assert np.allclose(-lap, k * k * f(r0), rtol=0, atol=2e-5 * np.abs(f(r0)).max() * k * k)
            assert abs(2 * b.half_lambda[alpha(l, 0, n, b.N)] - k * k) < 1e-14 * k * k


def test_real_harmonics_against_scipy():
    # real Y from scipy's complex harmonics (Condon-Shortley phase removed)
    lmax = 12
    b = Basis(4.0, lmax, 2, 6, 16, 30)
    theta = np.arccos(b.t)
    T, P = np.meshgrid(theta, b.phi, indexing="ij")
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            ours = b.theta[am][:, l - am][:, None] * b.phi_fn[:, m + lmax][None, :]
            yc = sp.sph_harm_y(l, am, T, P) * (-1) ** am
            if m == 0:
                ref = yc.real
            elif m > 0:
                ref = math.sqrt(2.0) * yc.real
            else:
                ref = math.sqrt(2.0) * yc.imag
            assert np.max(np.abs(ours - ref)) < 1e-12, (l, m)


def test_angular_orthonormality_exact_on_config_grid():
    # Gauss in cos(theta) with N_theta > lmax and N_phi > 2 lmax integrate Y Y' exactly
    for lmax, nt, nphi in [(10, 22, 42), (30, 60, 120)]:
        b = Basis(8.0, lmax, 1, 4, nt, nphi)
        L = lmax + 1
        Y = np.empty((nt * nphi, L * L))
        for l in range(L):
            for m in range(-l, l + 1):
                am = abs(m)
                Y[:, l * l + l + m] = (b.theta[am][:, l - am][:, None]
                                       * b.phi_fn[:, m + lmax][None, :]).ravel()
        w = (b.w_t[:, None] * np.full(nphi, b.w_phi)[None, :]).ravel()
        M = Y.T @ (w[:, None] * Y)
        assert np.max(np.abs(M - np.eye(L * L))) < 1e-13


@pytest.mark.parametrize("rule", ["gauss_legendre", "gauss_jacobi_r2"])
def test_discrete_orthonormality_resolved_quadrature(rule):
    # lmax = 10, N = 16, R = 8 (1936 functions) with 56 radial nodes: B^T W B = I to 1e-13
    b = Basis(8.0, 10, 16, 56, 22, 42, rule)
    B = b.synthesis_matrix()
    W = b.weights().ravel()
    M = B.T @ (W[:, None] * B)
    assert np.max(np.abs(M - np.eye(b.d))) < 1e-13


def test_config_quadrature_is_underresolved_radially():
    # with 32 radial nodes the same basis is not discretely orthonormal (documented reading)
    b = Basis(8.0, 10, 16, 32, 22, 42)
    B = b.synthesis_matrix()
    W = b.weights().ravel()
    M = B.T @ (W[:, None] * B)
    assert np.max(np.abs(M - np.eye(b.d))) > 1e-3


def test_forward_inverse_round_trip():
    b = Basis(7.0, 6, 8, 40, 14, 26)  # radial rule resolved for N = 8
    rng = np.random.default_rng(0)
    X = rng.standard_normal((b.d, 3))
    Y = b.forward_transform(b.inverse_transform(X))
    assert np.max(np.abs(Y - X)) < 1e-12


def test_transforms_match_explicit_synthesis_matrix():
    b = Basis(7.0, 5, 6, 14, 10, 20)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((b.d, 2))
    B = b.synthesis_matrix()
    f = b.inverse_transform(X).reshape(-1, 2)
    assert np.max(np.abs(f - B @ X)) < 1e-12
    g = rng.standard_normal((b.n_grid, 2))
    W = b.weights().ravel()
    ref = B.T @ (W[:, None] * g)
    got = b.forward_transform(g.reshape(b.n_r, b.n_theta, b.n_phi, 2))
    assert np.max(np.abs(got - ref)) < 1e-12 * np.abs(ref).max()


def test_index_map():
    N = 7
    seen = set()
    for l in range(5):
        for m in range(-l, l + 1):
            for n in range(N):
                seen.add(alpha(l, m, n, N))
    assert seen == set(range(25 * N))
    assert alpha(0, 0, 0, N) == 0 and alpha(1, -1, 0, N) == N and alpha(2, 2, 6, N) == 9 * N - 1
