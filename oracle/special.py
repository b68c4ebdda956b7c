"""Special functions and quadrature rules (FP64).

Test infrastructure only (see oracle/__init__.py).

The basis of Sec. 2.2.1 needs the spherical Bessel functions j_l and their zeros
b^n_{l+1/2} (eq. spherical_bessel_1, laplacian_eigenvalue), the normalised associated
Legendre functions without the Condon-Shortley phase (eq. spherical_harmonics_1 and its
footnote), and the Gauss rules of Sec. 2.2.2: Gauss points in cos(theta), and radial
Gauss-Jacobi points for the weight r^2 (or Gauss-Legendre points with r^2 put in the
weights). Sec. 3.4.2 names Halley's method for the zeros and Golub-Welsch for the Gauss
rules; any method that returns the same numbers to rounding is equivalent, and the
choices below are stated where they are made.
"""
from __future__ import annotations

import math

import numpy as np


def sph_bessel_j(l: int, x) -> np.ndarray:
    """Spherical Bessel function of the first kind j_l(x), integer l >= 0, real x >= 0.

    x > l: upward three-term recurrence j_{n+1} = (2n+1)/x j_n - j_{n-1} from
    j_0 = sin x / x and j_1 = sin x / x^2 - cos x / x (stable while n < x).
    x <= l: Miller's downward recurrence from order l+40 with per-point rescaling,
    normalised by least squares against the closed forms of j_0 and j_1 (they never
    vanish together).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.zeros_like(x)
    if l == 0:
        nz = x != 0.0
        out[~nz] = 1.0
        out[nz] = np.sin(x[nz]) / x[nz]
        return out
    up = x > l
    if np.any(up):
        xu = x[up]
        jm1 = np.sin(xu) / xu
        j = np.sin(xu) / (xu * xu) - np.cos(xu) / xu
        for n in range(1, l):
            jm1, j = j, (2 * n + 1) / xu * j - jm1
        out[up] = j
    down = (~up) & (x > 0.0)
    if np.any(down):
        xd = x[down]
        n_start = l + 40
        jp1 = np.zeros_like(xd)      # order n_start + 1
        j = np.full_like(xd, 1e-30)  # order n_start
        j_l = np.zeros_like(xd)
        for n in range(n_start, 0, -1):
            jm1 = (2 * n + 1) / xd * j - jp1   # order n - 1
            jp1, j = j, jm1
            if n - 1 == l:
                j_l = j.copy()
            big = np.abs(j) > 1e200
            if np.any(big):
                s = np.where(big, 1e-200, 1.0)
                j *= s
                jp1 *= s
                j_l *= s
        # j now holds order 0, jp1 order 1 (unnormalised)
        t0 = np.sin(xd) / xd
        t1 = np.sin(xd) / (xd * xd) - np.cos(xd) / xd
        nrm = np.maximum(np.abs(j), np.abs(jp1))
        u0, u1 = j / nrm, jp1 / nrm
        scale = (t0 * u0 + t1 * u1) / (u0 * u0 + u1 * u1)
        out[down] = (j_l / nrm) * scale
    return out


def sph_bessel_j_deriv(l: int, x) -> np.ndarray:
    """d/dx j_l(x) = j_{l-1}(x) - (l+1)/x j_l(x)  (l >= 1);  j_0' = -j_1."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    if l == 0:
        return -sph_bessel_j(1, x)
    return sph_bessel_j(l - 1, x) - (l + 1) / x * sph_bessel_j(l, x)


def _refine_root(l: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Bisection on brackets [a, b] (one sign change each) followed by Newton polish."""
    fa = sph_bessel_j(l, a)
    for _ in range(100):
        m = 0.5 * (a + b)
        fm = sph_bessel_j(l, m)
        left = np.sign(fm) == np.sign(fa)
        a = np.where(left, m, a)
        fa = np.where(left, fm, fa)
        b = np.where(left, b, m)
        if np.all(b - a <= 4.0 * np.finfo(np.float64).eps * b):
            break
    x = 0.5 * (a + b)
    for _ in range(2):
        f = sph_bessel_j(l, x)
        df = sph_bessel_j_deriv(l, x)
        x = x - f / df
    return x


def sph_bessel_zeros(lmax: int, nmax: int) -> np.ndarray:
    """z[l, n] = (n+1)-th positive zero of j_l (= b^n_{l+1/2}), l <= lmax, n < nmax.

    z_{0,n} = (n+1) pi. For l >= 1 the zeros of j_l and j_{l-1} interlace,
    z_{l-1,n} < z_{l,n} < z_{l-1,n+1}, so each bracket holds exactly one zero.
    """
    count = nmax + lmax + 1
    prev = np.pi * np.arange(1, count + 1, dtype=np.float64)
    z = np.zeros((lmax + 1, nmax))
    z[0] = prev[:nmax]
    for l in range(1, lmax + 1):
        cur = _refine_root(l, prev[:-1].copy(), prev[1:].copy())
        z[l] = cur[:nmax]
        prev = cur
    return z


def gauss_legendre(n: int):
    """Gauss-Legendre nodes (ascending) and weights on [-1, 1].

    Newton's method on P_n(x) from the asymptotic guesses cos(pi (i + 3/4)/(n + 1/2));
    P_n and P_n' by the three-term recurrence; w = 2 / ((1 - x^2) P_n'(x)^2).
    """
    i = np.arange(n, dtype=np.float64)
    x = np.cos(np.pi * (i + 0.75) / (n + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        if n == 1:
            p0, p1 = np.ones_like(x), x.copy()
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    if n == 1:
        p0 = np.ones_like(x)
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


def gauss_jacobi_0_2(n: int):
    """Gauss-Jacobi nodes (ascending) and weights on [-1, 1] for the weight (1 + x)^2.

    Golub-Welsch: the nodes are the eigenvalues of the symmetric tridiagonal Jacobi
    matrix of the orthonormal Jacobi polynomials (alpha = 0, beta = 2); the weights are
    mu_0 times the squared first components of the eigenvectors, mu_0 = 8/3.
    """
    al, be = 0.0, 2.0
    k = np.arange(n, dtype=np.float64)
    s = 2.0 * k + al + be
    diag = (be * be - al * al) / (s * (s + 2.0))
    kk = np.arange(1, n, dtype=np.float64)
    s1 = 2.0 * kk + al + be
    off = np.sqrt(4.0 * kk * (kk + al) * (kk + be) * (kk + al + be)
                  / (s1 * s1 * (s1 + 1.0) * (s1 - 1.0)))
    J = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    x, v = np.linalg.eigh(J)
    mu0 = 2.0 ** (al + be + 1.0) * math.gamma(al + 1) * math.gamma(be + 1) / math.gamma(al + be + 2)
    w = mu0 * v[0, :] ** 2
    return x, w


def norm_assoc_legendre(lmax: int, t) -> np.ndarray:
    """Theta[l, m, j] = c_lm P_l^m(t_j) for 0 <= m <= l <= lmax, zero for m > l.

    c_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) as in eq. spherical_harmonics_1, and
    P_l^m without the Condon-Shortley phase (footnote to the real-function symmetry in
    Sec. 2.2.1), so Theta_mm > 0 for |t| < 1. Standard normalised recurrences:
      Theta_00 = 1/sqrt(4 pi),
      Theta_mm = sqrt((2m+1)/(2m)) sqrt(1-t^2) Theta_{m-1,m-1},
      Theta_{m+1,m} = sqrt(2m+3) t Theta_mm,
      Theta_lm = a_lm (t Theta_{l-1,m} - b_lm Theta_{l-2,m}),
        a_lm = sqrt((4l^2-1)/(l^2-m^2)), b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
    """
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    st = np.sqrt(np.maximum(0.0, 1.0 - t * t))
    th = np.zeros((lmax + 1, lmax + 1, t.size))
    th[0, 0] = 1.0 / math.sqrt(4.0 * math.pi)
    for m in range(1, lmax + 1):
        th[m, m] = math.sqrt((2 * m + 1) / (2.0 * m)) * st * th[m - 1, m - 1]
    for m in range(0, lmax):
        th[m + 1, m] = math.sqrt(2 * m + 3) * t * th[m, m]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            th[l, m] = a * (t * th[l - 1, m] - b * th[l - 2, m])
    return th
