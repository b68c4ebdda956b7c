"""Pins for oracle/hamiltonian.py: kinetic diagonal, brute-force dense H, Hermiticity,
constant and radial potentials, coupling selection rules, the 3-D harmonic oscillator
spectrum, the projector pair, and planted mistakes that the pins must catch."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.basis import Basis, alpha, basis_for
from oracle.hamiltonian import Hamiltonian


def _small():
    w = W.small_cluster()
    b = basis_for(w)
    return w, b, Hamiltonian(b, w.potential_at(b.points()))


def test_zero_potential_gives_kinetic_diagonal():
    b = Basis(6.0, 5, 7, 16, 12, 22)
    H = Hamiltonian(b, np.zeros(b.n_grid))
    X = W.gaussian_block(11, b.d, 4)
    assert np.array_equal(H.apply(X), b.half_lambda[:, None] * X)


def test_separable_matches_dense_brute_force():
    w, b, H = _small()
    X = w.x_block()
    ref = H.dense() @ X
    got = H.apply(X)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()


def test_hermiticity():
    w, b, H = _small()
    u = W.gaussian(21, b.d)
    v = W.gaussian(22, b.d)
    Hd = H.dense()
    assert np.max(np.abs(Hd - Hd.T)) < 1e-14 * np.abs(Hd).max()
    lhs = u @ H.apply(v)
    rhs = H.apply(u) @ v
    assert abs(lhs - rhs) < 1e-14 * np.linalg.norm(Hd, 2) * np.linalg.norm(u) * np.linalg.norm(v)


def test_constant_potential_shifts_spectrum():
    # resolved radial quadrature: B^T W B = I, so V = v0 gives H = 1/2 Lambda + v0 I
    b = Basis(6.0, 4, 6, 40, 10, 20)
    v0 = -0.731
    H = Hamiltonian(b, np.full(b.n_grid, v0))
    Hd = H.dense()
    assert np.max(np.abs(Hd - np.diag(b.half_lambda + v0))) < 1e-13


def test_centred_radial_potential_is_block_diagonal_in_lm():
    b = Basis(6.0, 4, 6, 30, 10, 20)
    r = np.linalg.norm(b.points(), axis=1)
    H = Hamiltonian(b, np.exp(-r) * 3.0 - 1.0)
    Hd = H.dense()
    N = b.N
    for l in range(b.L):
        for m in range(-l, l + 1):
            a = alpha(l, m, 0, N)
            blk = Hd[a:a + N, :].copy()
            blk[:, a:a + N] = 0.0
            assert np.max(np.abs(blk)) < 1e-13
            # the (l, m) block does not depend on m
            a0 = alpha(l, 0, 0, N)
            assert np.max(np.abs(Hd[a:a + N, a:a + N] - Hd[a0:a0 + N, a0:a0 + N])) < 1e-13


def test_z_coupling_selection_rule():
    # V = f(r) z = f(r) r cos(theta) ~ Y_10 couples only l <-> l +- 1 at equal m
    b = Basis(6.0, 5, 5, 30, 12, 24)
    p = b.points()
    r = np.linalg.norm(p, axis=1)
    H = Hamiltonian(b, np.exp(-0.3 * r) * p[:, 2])
    Hd = H.dense()
    np.fill_diagonal(Hd, Hd.diagonal() - b.half_lambda)
    N = b.N
    for l in range(b.L):
        for m in range(-l, l + 1):
            for l2 in range(b.L):
                for m2 in range(-l2, l2 + 1):
                    blk = Hd[alpha(l, m, 0, N):alpha(l, m, 0, N) + N,
                             alpha(l2, m2, 0, N):alpha(l2, m2, 0, N) + N]
                    allowed = (m == m2) and abs(l - l2) == 1
                    if not allowed:
                        assert np.max(np.abs(blk)) < 1e-13, (l, m, l2, m2)


def _ho_levels(n):
    # 3-D isotropic oscillator, omega = 1: E = 2 n_r + l + 3/2, degeneracy 2l+1
    lev = []
    for nr in range(10):
        for l in range(20):
            lev += [2 * nr + l + 1.5] * (2 * l + 1)
    return np.sort(lev)[:n]


def test_harmonic_oscillator_spectrum_dense():
    w = W.harmonic_oscillator_ball()
    b = basis_for(w)
    H = Hamiltonian(b, w.potential_at(b.points()))
    ev = np.linalg.eigvalsh(H.dense())
    assert np.max(np.abs(ev[:10] - _ho_levels(10))) < 1e-6
    assert np.max(np.abs(ev[:10] - _ho_levels(10))) < 1e-11  # observed ~1e-13
    golden = np.loadtxt(__file__.replace("test_oracle_hamiltonian.py", "golden/ho_levels.txt"))
    assert np.max(np.abs(ev[:10] - golden[:10])) < 1e-6


def test_kb_projector_pair():
    b = Basis(6.0, 4, 8, 40, 10, 20)
    atoms = np.array([[0.0, 0.0, 0.0], [1.0, -0.5, 0.7]])
    pg, h = W.kb_projector_values(b.points(), atoms, rc=1.0)
    v = np.zeros(b.n_grid)
    Hloc = Hamiltonian(b, v)
    Hkb = Hamiltonian(b, v, pg, h)
    X = W.gaussian_block(5, b.d, 3)
    diff = Hkb.apply(X) - Hloc.apply(X)
    P = Hkb.P
    ref = sum(h[i] * np.outer(P[:, i], P[:, i] @ X) for i in range(len(h)))
    assert np.max(np.abs(diff - ref)) < 1e-13 * np.abs(ref).max()
    # a Gaussian s projector at the origin has only l = 0 coefficients; p_z only (1, 0)
    s_coef = P[:, 0]
    pz_coef = P[:, 3]
    N = b.N
    assert np.max(np.abs(s_coef[N:])) < 1e-13 * np.abs(s_coef).max()
    mask = np.ones(b.d, bool)
    mask[alpha(1, 0, 0, N):alpha(1, 0, 0, N) + N] = False
    assert np.max(np.abs(pz_coef[mask])) < 1e-13 * np.abs(pz_coef).max()
    # expansion captures (almost) the whole unit norm of the projector
    assert abs(np.sum(s_coef ** 2) - 1.0) < 1e-3


# ------------------------------------------------------------------ planted mistakes
# Each test plants a plausible mistake in a copy of the oracle (on the CPU) and checks
# that at least one of the pins above would fail.

def test_planted_missing_sqrt2_breaks_orthonormality():
    b = Basis(6.0, 4, 1, 4, 10, 20)
    b.phi_fn[:, b.lmax + 1:] /= math.sqrt(2.0)  # drop sqrt2 on the cos functions
    L = b.L
    Y = np.empty((b.n_theta * b.n_phi, L * L))
    for l in range(L):
        for m in range(-l, l + 1):
            Y[:, l * l + l + m] = (b.theta[abs(m)][:, l - abs(m)][:, None]
                                   * b.phi_fn[:, m + b.lmax][None, :]).ravel()
    w = (b.w_t[:, None] * np.full(b.n_phi, b.w_phi)[None, :]).ravel()
    assert np.max(np.abs(Y.T @ (w[:, None] * Y) - np.eye(L * L))) > 0.1


def test_planted_dropped_kinetic_breaks_ho():
    w = W.harmonic_oscillator_ball()
    b = basis_for(w)
    b.half_lambda = 0.5 * b.half_lambda  # wrong factor on the Laplacian eigenvalue
    H = Hamiltonian(b, w.potential_at(b.points()))
    ev = np.linalg.eigvalsh(H.dense())
    assert np.max(np.abs(ev[:10] - _ho_levels(10))) > 1e-2


def test_planted_reversed_theta_nodes_break_scipy_harmonics():
    from scipy import special as sp
    b = Basis(4.0, 6, 1, 4, 12, 24)
    b.theta[1] = b.theta[1][::-1, :].copy()  # m = 1 rows in the wrong node order
    T, P = np.meshgrid(np.arccos(b.t), b.phi, indexing="ij")
    l, m = 2, 1
    ours = b.theta[m][:, l - m][:, None] * b.phi_fn[:, m + b.lmax][None, :]
    ref = math.sqrt(2.0) * (sp.sph_harm_y(l, m, T, P) * (-1) ** m).real
    assert np.max(np.abs(ours - ref)) > 0.1


def test_hydrogen_like_l0_levels_decrease_toward_exact():
    """V = -1/r in the l = 0 subspace (R = 20, resolved radial rule): the two lowest levels
    are variational upper bounds that decrease monotonically with the number of radial
    functions toward the hydrogen levels -1/2 and -1/8 Ha (slow, polynomial convergence: the
    cusp at the origin)."""
    from oracle.basis import Basis
    prev = None
    for N in (8, 16, 24, 32):
        b = Basis(20.0, 0, N, n_r=4 * N + 16, n_theta=2, n_phi=2)
        r = np.linalg.norm(b.points(), axis=1)
        lam = np.linalg.eigvalsh(Hamiltonian(b, -1.0 / r).dense())[:2]
        assert lam[0] > -0.5 and lam[1] > -0.125
        if prev is not None:
            assert lam[0] < prev[0] and lam[1] < prev[1]
        prev = lam
    assert prev[0] < -0.49 and prev[1] < -0.123


def test_displaced_atom_converges_to_centred_atom():
    """Translation: one erf pseudo-atom (Z = 4, rc = 0.8) displaced 1.5 bohr along z in a ball
    of radius 10. Its lowest level is an upper bound that approaches, monotonically in lmax,
    the level of the same atom at the centre (converged in N with l = 0 alone), to 1e-4 Ha at
    lmax 10."""
    from oracle.basis import Basis

    def lowest(lmax, N, shift):
        b = Basis(10.0, lmax, N, n_r=2 * N + 24, n_theta=2 * lmax + 2, n_phi=4 * lmax + 4)
        v = W.erf_cluster_potential(b.points(), np.array([[0.0, 0.0, shift]]), 4.0, 0.8)
        return np.linalg.eigvalsh(Hamiltonian(b, v).dense())[0]

    centre = lowest(0, 32, 0.0)
    assert abs(centre - lowest(0, 24, 0.0)) < 1e-6  # converged in N
    shifted = [lowest(lmax, 16, 1.5) for lmax in (6, 8, 10)]
    assert shifted[0] > shifted[1] > shifted[2] > centre - 1e-9
    assert shifted[2] - centre < 1e-4
