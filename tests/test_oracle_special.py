"""Pins for oracle/special.py: closed forms, an independent library (scipy.special,
numpy.polynomial) and mathematical invariants. These tests need no GPU."""
import math

import numpy as np
import pytest
from scipy import special as sp

from oracle.special import (gauss_jacobi_0_2, gauss_legendre, norm_assoc_legendre,
                            sph_bessel_j, sph_bessel_zeros)


def test_j0_j1_closed_forms():
    x = np.linspace(1.0, 200.0, 5001)  # the j_1 closed form cancels for x << 1
    assert np.allclose(sph_bessel_j(0, x), np.sin(x) / x, rtol=0, atol=1e-16)
    j1 = np.sin(x) / x ** 2 - np.cos(x) / x
    assert np.max(np.abs(sph_bessel_j(1, x) - j1)) < 1e-15
    assert sph_bessel_j(0, np.array([0.0]))[0] == 1.0
    assert sph_bessel_j(3, np.array([0.0]))[0] == 0.0


@pytest.mark.parametrize("l", [0, 1, 2, 5, 10, 17, 30, 45, 61])
def test_jl_against_scipy(l):
    x = np.concatenate([np.logspace(-5, 0, 40), np.linspace(0.3, 420.0, 3000)])
    a = sph_bessel_j(l, x)
    b = sp.spherical_jn(l, x)
    env = np.maximum(np.abs(b), np.maximum.accumulate(np.abs(b)[::-1])[::-1])  # local envelope
    env = np.maximum(env, 1e-300)
    # relative to the local envelope: tiny values near zeros are judged absolutely
    assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-12 * env.max())) < 1e-9
    big = np.abs(b) > 1e-3 * np.abs(b).max()
    assert np.max(np.abs(a[big] - b[big]) / np.abs(b[big])) < 1e-11


def test_jl_small_x_series():
    # j_l(x) ~ x^l/(2l+1)!! (1 - x^2/(2(2l+3))) for tiny x
    for l in [1, 4, 9, 20]:
        x = np.array([1e-4, 3e-3])
        dfac = math.prod(range(1, 2 * l + 2, 2))
        ref = x ** l / dfac * (1 - x * x / (2 * (2 * l + 3)))
        assert np.allclose(sph_bessel_j(l, x), ref, rtol=1e-12, atol=0)


def test_zeros_l0_exact_and_l1_transcendental():
    z = sph_bessel_zeros(3, 40)
    assert np.max(np.abs(z[0] - np.pi * np.arange(1, 41))) < 1e-13
    # zeros of j_1 solve tan x = x
    assert np.max(np.abs(np.tan(z[1]) - z[1]) / z[1]) < 1e-11


def test_zeros_interlace_and_scipy_sign_changes():
    lmax, nmax = 40, 60
    z = sph_bessel_zeros(lmax, nmax)
    assert np.all(np.diff(z, axis=1) > 0)
    for l in range(1, lmax + 1):
        assert np.all(z[l - 1] < z[l])
        assert np.all(z[l, :-1] < z[l - 1, 1:])
    for l in [0, 3, 17, 40]:
        # scipy's j_l changes sign across each zero and is ~0 at it
        eps = 1e-9
        assert np.all(sp.spherical_jn(l, z[l] - eps) * sp.spherical_jn(l, z[l] + eps) < 0)
        assert np.max(np.abs(sp.spherical_jn(l, z[l]))) < 1e-14
        # first zero of j_l is above l (and below l + 2 l^(1/3) + 3 for l >= 1, McMahon)
        assert z[l, 0] > l


def test_gauss_legendre_against_numpy_and_exactness():
    for n in [1, 2, 7, 22, 60, 120]:
        x, w = gauss_legendre(n)
        xn, wn = np.polynomial.legendre.leggauss(n)
        assert np.max(np.abs(x - xn)) < 1e-14 and np.max(np.abs(w - wn)) < 1e-13
        assert abs(w.sum() - 2.0) < 1e-13
        for p in range(0, 2 * n):
            exact = (1 - (-1) ** (p + 1)) / (p + 1)
            assert abs(np.sum(w * x ** p) - exact) < 1e-12


def test_gauss_jacobi_r2_against_scipy_and_exactness():
    for n in [1, 5, 32, 96]:
        x, w = gauss_jacobi_0_2(n)
        xr, wr = sp.roots_jacobi(n, 0.0, 2.0)
        assert np.max(np.abs(x - xr)) < 1e-13 and np.max(np.abs(w - wr)) < 1e-12
        # int_{-1}^{1} (1+x)^2 x^p dx exact for p <= 2n-1
        for p in range(0, min(2 * n, 40)):
            t = np.polynomial.polynomial
            poly = t.polymul([1, 2, 1], [0] * p + [1])
            integ = t.polyint(poly)
            exact = t.polyval(1.0, integ) - t.polyval(-1.0, integ)
            assert abs(np.sum(w * x ** p) - exact) < 1e-11 * max(1.0, abs(exact))


def test_norm_assoc_legendre_against_scipy():
    t = np.linspace(-0.999, 0.999, 41)
    lmax = 40
    th = norm_assoc_legendre(lmax, t)
    for l in range(lmax + 1):
        for m in range(l + 1):
            c = math.sqrt((2 * l + 1) / (4 * math.pi)
                          * math.exp(math.lgamma(l - m + 1) - math.lgamma(l + m + 1)))
            ref = c * sp.lpmv(m, l, t) * (-1) ** m  # scipy includes the Condon-Shortley phase
            assert np.max(np.abs(th[l, m] - ref)) < 1e-12
    assert np.all(th[5, 5] > 0)  # no Condon-Shortley phase


def test_norm_assoc_legendre_orthonormal_on_gauss_grid():
    lmax = 30
    t, w = gauss_legendre(lmax + 1)
    th = norm_assoc_legendre(lmax, t)
    for m in range(lmax + 1):
        P = th[m:, m, :]  # (L-m, nt)
        M = 2 * np.pi * (P * w[None, :]) @ P.T
        assert np.max(np.abs(M - np.eye(lmax + 1 - m))) < 1e-13
