"""Pins of the SCF oracle (oracle/scf.py): the Hartree kernel against the Dirichlet
eigenfunction solution and an analytic Gaussian charge, the LDA potential as the
derivative of the energy density, Fermi-Dirac occupations, Anderson mixing on a linear
fixed-point problem, the density of a single basis function by brute force, the light
atoms of the paper's table, and planted mistakes that the pins must catch."""
import math
import pathlib

import numpy as np
import pytest

import workloads as W
from oracle import scf
from oracle.basis import Basis, alpha, basis_for

GOLDEN = pathlib.Path(__file__).parent / "golden" / "light_atoms_lda.txt"


def _gauss_charge(b, a, sig, Q):
    from scipy.special import erf
    xyz = b.points()
    d = np.linalg.norm(xyz - np.asarray(a)[None, :], axis=1)
    rho = Q * (2 * math.pi * sig ** 2) ** -1.5 * np.exp(-d ** 2 / (2 * sig ** 2))
    pot = Q * erf(d / (math.sqrt(2.0) * sig)) / d
    shape = (b.n_r, b.n_theta, b.n_phi)
    return rho.reshape(shape), pot.reshape(shape)


# ------------------------------------------------------------------ Hartree
def test_zeta_equals_dirichlet_solution_plus_multipole():
    """Z_ln of eq. zeta_definition (quadrature of the Laplace-expansion kernel) against a
    second derivation: R_ln is a Dirichlet eigenfunction of -Lap with eigenvalue k^2, so the
    potential of the charge R_ln Y_lm is 4 pi/k^2 R_ln Y_lm plus the harmonic r^l Y_lm term
    that matches the exterior multipole 4 pi/(2l+1) q / R^(l+1) at r = R, with
    q = int_0^R r^(l+2) R_ln = sqrt(2/R^3) R^(l+2)/k (from d/dx[x^(l+2) j_(l+1)] = x^(l+2) j_l).
    Hence Z_ln(r) = (2l+1)/k^2 R_ln(r) + sqrt(2/R^3) r^l R^(1-l) / k."""
    b = Basis(8.0, 6, 8, 20, 14, 28)
    zt = scf.zeta_tables(b)
    for l in range(b.L):
        for n in range(b.N):
            k = b.z[l, n] / b.R
            closed = ((2 * l + 1) / k ** 2 * b.radial[l][:, n]
                      + math.sqrt(2.0 / b.R ** 3) * b.r ** l * b.R ** (1 - l) / k)
            assert np.max(np.abs(zt[l][:, n] - closed)) <= 1e-13 * np.max(np.abs(closed))


def test_hartree_of_gaussian_charge_is_erf_potential():
    """An off-centre Gaussian charge Q (2 pi s^2)^-3/2 exp(-|x-a|^2/2s^2) has the potential
    Q erf(|x-a|/(sqrt2 s))/|x-a| and the self-energy Q^2/(2 sqrt(pi) s)."""
    b = Basis(8.0, 12, 24, 48, 26, 50)
    rho, pot = _gauss_charge(b, (0.5, -0.3, 0.4), 1.0, 3.0)
    vh = scf.hartree(b, rho)
    assert np.max(np.abs(vh - pot)) <= 1e-10 * np.max(np.abs(pot))
    eh = 0.5 * scf.integral(b, rho, vh)
    assert abs(eh - 9.0 / (2.0 * math.sqrt(math.pi))) <= 1e-10


def test_hartree_is_symmetric():
    """int rho1 V_H[rho2] = int rho2 V_H[rho1] (symmetric Green's function) for densities in
    the span of the basis, on a grid that resolves the basis products."""
    b = Basis(7.0, 4, 6, 40, 12, 22)
    c = W.gaussian_block(43, b.d, 2)
    r1 = b.inverse_transform(c[:, :1])[..., 0]
    r2 = b.inverse_transform(c[:, 1:])[..., 0]
    zt = scf.zeta_tables(b)
    a = scf.integral(b, r1, scf.hartree(b, r2, zt))
    d = scf.integral(b, r2, scf.hartree(b, r1, zt))
    assert abs(a - d) <= 1e-12 * max(abs(a), 1.0)


# ------------------------------------------------------------------ LDA
def test_lda_potential_is_derivative_of_energy_density():
    rho = np.logspace(-7, 3, 200)
    e, v = scf.lda_xc(rho)
    h = 1e-6
    ep, _ = scf.lda_xc(rho * (1 + h))
    em, _ = scf.lda_xc(rho * (1 - h))
    fd = (rho * (1 + h) * ep - rho * (1 - h) * em) / (2 * h * rho)
    assert np.max(np.abs(fd - v) / np.abs(v)) <= 1e-8


def test_lda_exchange_and_correlation_closed_forms():
    """Slater exchange of the uniform gas, eps_x = -(3/(4 pi)) (9 pi/4)^(1/3) / rs; the
    Perdew-Zunger fit is continuous at rs = 1 (both branches agree to 5e-5 in eps_c and
    v_c), and vanishes with the density."""
    rs = np.array([0.5, 1.0, 2.0, 5.0])
    rho = 3.0 / (4.0 * math.pi * rs ** 3)
    e_x_only = -(3.0 / (4.0 * math.pi)) * (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
    e, _ = scf.lda_xc(rho)
    ec = e - e_x_only
    assert np.all(ec < 0) and np.all(np.diff(ec) > 0)  # correlation negative, weaker at low density
    # continuity of both branches at rs = 1
    hi = scf.PZ_GAMMA / (1 + scf.PZ_BETA1 + scf.PZ_BETA2)
    lo = scf.PZ_B + scf.PZ_D
    assert abs(hi - lo) <= 5e-5
    vhi = hi * (1 + 7.0 / 6.0 * scf.PZ_BETA1 + 4.0 / 3.0 * scf.PZ_BETA2) / (1 + scf.PZ_BETA1 + scf.PZ_BETA2)
    vlo = scf.PZ_B - scf.PZ_A / 3.0 + (2 * scf.PZ_D - scf.PZ_C) / 3.0
    assert abs(vhi - vlo) <= 5e-5
    e0, v0 = scf.lda_xc(np.array([0.0, -1e-3]))
    assert np.all(e0 == 0) and np.all(v0 == 0)


# ------------------------------------------------------------------ occupations
def test_fermi_occupations():
    lam = np.array([-1.0, -0.5, -0.5, 0.2, 0.9])
    f, mu, S = scf.fermi_occupations(lam, 4.0, 1e-3)
    assert abs(f.sum() - 2.0) <= 1e-12
    # two electrons fill the lowest level; the degenerate pair shares the other two
    assert abs(f[0] - 1.0) <= 1e-12 and abs(f[1] - 0.5) <= 1e-9 and abs(f[2] - 0.5) <= 1e-9
    assert abs(mu - (-0.5)) <= 1e-9
    assert abs(S - 4.0 * math.log(2.0)) <= 1e-6
    f2, _, _ = scf.fermi_occupations(lam, 3.0, 0.05)
    assert abs(f2.sum() - 1.5) <= 1e-12 and np.all(np.diff(f2) <= 1e-15)


# ------------------------------------------------------------------ mixing
def test_anderson_solves_linear_fixed_point_in_n_plus_one_steps():
    """For g(x) = A x + c with full history, Anderson mixing spans the Krylov space of the
    residuals (it is equivalent to GMRES), so it reaches the fixed point of an n-dimensional
    problem after at most n + 1 steps."""
    rng = np.random.default_rng(5)
    n = 6
    M = rng.standard_normal((n, n))
    A = 0.4 * M / np.linalg.norm(M, 2)
    c = rng.standard_normal(n)
    xstar = np.linalg.solve(np.eye(n) - A, c)
    w = rng.uniform(0.5, 1.5, n)
    mix = scf.Anderson(w, beta=0.3)
    x = np.zeros(n)
    for _ in range(n + 2):
        x = mix.mix(x, A @ x + c)
    assert np.max(np.abs(x - xstar)) <= 1e-9
    # linear mixing alone (history 0) is far from converged after the same number of steps
    lin = scf.Anderson(w, beta=0.3, history=0)
    y = np.zeros(n)
    for _ in range(n + 2):
        y = lin.mix(y, A @ y + c)
    assert np.max(np.abs(y - xstar)) > 1e-3


# ------------------------------------------------------------------ density
def test_density_of_one_basis_function_by_brute_force():
    """rho = 2 f F_lmn(x)^2 for X = e_alpha: R_ln from scipy's spherical_jn, Y_lm (real,
    no Condon-Shortley phase) from scipy's associated Legendre functions."""
    from scipy.special import lpmv, spherical_jn
    b = Basis(6.0, 4, 5, 12, 10, 20)
    for (l, m, n) in [(0, 0, 0), (2, -1, 3), (3, 2, 1), (4, -4, 4)]:
        X = np.zeros((b.d, 1))
        X[alpha(l, m, n, b.N), 0] = 1.0
        rho = scf.density(b, X, np.array([0.7]))
        xyz = b.points()
        r = np.linalg.norm(xyz, axis=1)
        t = xyz[:, 2] / r
        ph = np.arctan2(xyz[:, 1], xyz[:, 0])
        k = b.z[l, n] / b.R
        Rl = math.sqrt(2.0 / b.R ** 3) * spherical_jn(l, k * r) / spherical_jn(l + 1, b.z[l, n])
        am = abs(m)
        c = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
        P = (-1) ** am * lpmv(am, l, t)  # remove scipy's Condon-Shortley phase
        Y = c * P * (1.0 if m == 0 else math.sqrt(2.0) * (np.cos(am * ph) if m > 0 else np.sin(am * ph)))
        ref = 2 * 0.7 * (Rl * Y) ** 2
        assert np.max(np.abs(rho.ravel() - ref)) <= 1e-12 * np.max(ref)


def test_density_integrates_to_electron_count_at_resolved_quadrature():
    b = Basis(8.0, 4, 8, 40, 12, 22)  # radial rule resolves products of the N = 8 functions
    X = np.linalg.qr(W.gaussian_block(41, b.d, 5))[0]
    occ = np.array([1.0, 1.0, 0.8, 0.5, 0.1])
    rho = scf.density(b, X, occ)
    assert abs(scf.integral(b, rho) - 2.0 * occ.sum()) <= 1e-12


# ------------------------------------------------------------------ SCF
def _light_atom(Z, ne, N):
    b = Basis(10.0 if Z > 1 else 12.0, 0, N, 2 * N, 1, 1, "gauss_jacobi_r2")
    r = np.linalg.norm(b.points(), axis=1)
    rho0 = ne * (Z ** 3 / math.pi) * np.exp(-2 * Z * r)
    return scf.scf(b, -Z / r, float(ne), rho0, 2, kT=1e-6, beta=0.5, tol=1e-10, max_iter=100)


def _golden():
    rows = []
    for line in GOLDEN.read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            el, z, ne, e = line.split()
            rows.append((el, float(z), float(ne), float(e)))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: r[0])
def test_light_atoms_match_paper_table(row):
    """All-electron LDA SCF of H and He (Coulomb nucleus, l = 0 basis, 80 / 120 radial
    functions) against the paper's table; the Coulomb cusp converges slowly in N, as the
    paper notes, so the tolerance is 2e-3 Ha (the spread of the table's own columns)."""
    el, Z, ne, e_ref = row
    out = _light_atom(Z, ne, 80 if Z == 1 else 120)
    assert out["converged"]
    assert abs(out["energy"] - e_ref) <= 2e-3


def test_scf_small_cluster_converges_and_energy_identity():
    """An erf cluster of two Z=2 pseudo-atoms: the SCF converges (|dE| <= 1e-9 Ha), the
    density holds the electron count on a resolved grid, and the band-energy form of the
    free energy equals the term-by-term functional (kinetic energy from the coefficients)."""
    b = Basis(7.0, 4, 8, 24, 12, 24)
    atoms = np.array([[0.0, 0.0, 0.7], [0.0, 0.0, -0.7]])
    vext = W.erf_cluster_potential(b.points(), atoms, Z=2.0, rc=0.8)
    rho0 = W.gaussian_atom_density(b.points(), atoms, Z=2.0, sigma=1.0)
    out = scf.scf(b, vext, 4.0, rho0, 4, kT=1e-3, beta=0.3, tol=1e-9, max_iter=80)
    assert out["converged"]
    shape = (b.n_r, b.n_theta, b.n_phi)
    e_dir = scf.direct_energy(b, out["X"], out["occ"], out["entropy"], 1e-3, out["rho"],
                              vext.reshape(shape), out["vh"], out["exc"])
    assert abs(out["energy"] - e_dir) <= 1e-8


# ------------------------------------------------------------------ planted mistakes
def test_planted_missing_spin_factor_breaks_helium():
    orig = scf.density
    try:
        scf.density = lambda b, X, occ: 0.5 * orig(b, X, occ)  # rho without the factor 2
        out = _light_atom(2.0, 2.0, 60)
    finally:
        scf.density = orig
    assert abs(out["energy"] - (-2.834)) > 0.1


def test_planted_hartree_without_2l_plus_1_breaks_gaussian_pin():
    b = Basis(8.0, 12, 24, 48, 26, 50)
    rho, pot = _gauss_charge(b, (0.5, -0.3, 0.4), 1.0, 3.0)
    zt = scf.zeta_tables(b)
    for l in range(b.L):
        zt[l] = zt[l] * (2 * l + 1)  # planted: 4 pi instead of 4 pi/(2l+1)
    vh = scf.hartree(b, rho, zt)
    assert np.max(np.abs(vh - pot)) > 1e-3 * np.max(np.abs(pot))


def test_planted_wrong_exchange_factor_breaks_derivative_pin():
    rho = np.logspace(-3, 1, 20)
    e, v = scf.lda_xc(rho)
    ex = -0.75 * (3.0 * rho / math.pi) ** (1.0 / 3.0)
    v_bad = v - 4.0 / 3.0 * ex + ex  # planted: v_x = eps_x
    h = 1e-6
    ep, _ = scf.lda_xc(rho * (1 + h))
    em, _ = scf.lda_xc(rho * (1 - h))
    fd = (rho * (1 + h) * ep - rho * (1 - h) * em) / (2 * h * rho)
    assert np.max(np.abs(fd - v_bad) / np.abs(v_bad)) > 1e-2
