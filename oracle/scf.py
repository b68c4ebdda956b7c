"""Self-consistent field pieces (FP64): electron density, Hartree potential, LDA exchange and
correlation, Fermi-Dirac occupations, Anderson mixing of the effective potential, and the
SCF loop built from them.

Test infrastructure only (see oracle/__init__.py).

- Sec. 2.1, eq. density_expression: rho = 2 sum_i f_i |phi_i|^2. The system is
  spin-unpolarised and 0 <= f_i <= 1.
- Sec. 2.2.5: the density is evaluated on the grid through inverse basis transforms of the
  orbitals (the transform method, not the coupling-coefficient sum).
- Sec. 2.3.1 (Hartree potential).
  - tau = forward transform of rho in the wavefunction basis. This is the dualing
    approximation: the density uses the orbitals' basis.
  - V_H(x) = sum_lmn 4 pi/(2l+1) tau_lmn Y_lm(x) Z_ln(r) (eq. hartree_calc1). This is an
    inverse transform with the functions Z_ln in place of R_ln.
  - Z_ln(r) = int_0^R r_<^l / r_>^(l+1) R_ln(r') r'^2 dr' (eq. zeta_definition), taken here
    by composite Gauss-Legendre quadrature split at r. The paper tabulates the same integral
    and splines it.
- Sec. 2.1 (LDA): Slater exchange plus the Perdew-Zunger (1981) parametrisation of the
  Ceperley-Alder correlation energy, unpolarised. eps is per electron; v = d(rho eps)/d rho.
- Sec. 3.4.1: Fermi-Dirac occupations, with the Fermi level fixed by the electron count
  (eq. Fermi_constraint, Brent's method); and Anderson mixing of the effective potential with
  linear parameter beta. The mixing inner product is the grid quadrature.
"""
from __future__ import annotations

import copy
import math

import numpy as np

from .basis import Basis
from .hamiltonian import Hamiltonian
from .special import gauss_legendre, sph_bessel_j

FOUR_PI = 4.0 * math.pi


# ------------------------------------------------------------------------------ density
def density(basis: Basis, X: np.ndarray, occ: np.ndarray) -> np.ndarray:
    """rho[k, j, q] = 2 sum_s occ_s psi_s(x_kjq)^2 with psi_s the inverse transform of X[:, s]
    (eq. density_expression; Sec. 2.2.5)."""
    X = np.asarray(X, dtype=np.float64)
    f = basis.inverse_transform(X)
    return 2.0 * np.einsum("kjqs,s->kjq", f * f, np.asarray(occ, dtype=np.float64))


def integral(basis: Basis, *fs: np.ndarray) -> float:
    """Grid quadrature of the pointwise product of grid functions: sum_g W_g prod f(x_g)."""
    p = basis.weights().copy()
    for f in fs:
        p = p * np.asarray(f, dtype=np.float64).reshape(p.shape)
    return float(p.sum())


# ------------------------------------------------------------------------------ Hartree
def zeta_tables(basis: Basis, panels_per_unit: float = 1.0, q: int = 16) -> list:
    """Z_ln(r_k) for every l, n and radial node (eq. zeta_definition):

        Z_ln(r) = r^-(l+1) int_0^r t^(l+2) R_ln(t) dt + r^l int_r^R t^(1-l) R_ln(t) dt.

    The interval [0, R] is cut at every node r_k. Each piece is split into sub-panels of
    length about 1/(panels_per_unit k_ln), each with q Gauss-Legendre points, and cumulative
    sums give both integrals at every node."""
    R, L, N = basis.R, basis.L, basis.N
    r = basis.r
    order = np.argsort(r)
    rs = r[order]
    edges = np.concatenate([[0.0], rs, [R]])
    xg, wg = gauss_legendre(q)
    tables = []
    for l in range(L):
        tab = np.empty((basis.n_r, N))
        for n in range(N):
            k = basis.z[l, n] / R
            norm = math.sqrt(2.0 / R ** 3) / sph_bessel_j(l + 1, basis.z[l, n])[0]
            lower = np.empty(len(edges) - 1)  # integral of t^(l+2) R over each piece
            upper = np.empty(len(edges) - 1)  # integral of t^(1-l) R over each piece
            for i in range(len(edges) - 1):
                a, b = edges[i], edges[i + 1]
                if b <= a:
                    lower[i] = upper[i] = 0.0
                    continue
                m = max(1, int(math.ceil((b - a) * k * panels_per_unit)))
                sub = np.linspace(a, b, m + 1)
                h = 0.5 * (sub[1:] - sub[:-1])
                c = 0.5 * (sub[1:] + sub[:-1])
                t = (c[:, None] + h[:, None] * xg[None, :]).ravel()
                w = (h[:, None] * wg[None, :]).ravel()
                Rt = norm * sph_bessel_j(l, k * t)
                lower[i] = np.sum(w * t ** (l + 2) * Rt)
                upper[i] = np.sum(w * t ** (1 - l) * Rt)
            cum_low = np.cumsum(lower)           # int_0^{edges[i+1]}
            tail_up = np.cumsum(upper[::-1])[::-1]  # int_{edges[i]}^R
            # node rs[i] = edges[i + 1]
            zs = np.empty(basis.n_r)
            for i in range(basis.n_r):
                ri = rs[i]
                zs[i] = cum_low[i] / ri ** (l + 1) + ri ** l * tail_up[i + 1]
            tab[order, n] = zs
        tables.append(tab)
    return tables


def hartree(basis: Basis, rho: np.ndarray, zeta: list | None = None) -> np.ndarray:
    """V_H on the grid from the grid density (Sec. 2.3.1): tau = forward transform of rho,
    then the inverse-transform-like sum of eq. hartree_calc1 with Z_ln and 4 pi/(2l+1)."""
    rho = np.asarray(rho, dtype=np.float64).reshape(basis.n_r, basis.n_theta, basis.n_phi)
    tau = basis.forward_transform(rho[..., None])[:, 0]
    L, N = basis.L, basis.N
    c = np.empty_like(tau)
    for l in range(L):
        a0, a1 = l * l * N, (l + 1) * (l + 1) * N
        c[a0:a1] = FOUR_PI / (2 * l + 1) * tau[a0:a1]
    zb = copy.copy(basis)
    zb.radial = zeta if zeta is not None else zeta_tables(basis)
    return zb.inverse_transform(c[:, None])[..., 0]


# ------------------------------------------------------------------------------ LDA
# Perdew & Zunger, Phys. Rev. B 23, 5048 (1981), unpolarised fit of Ceperley-Alder
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def lda_xc(rho: np.ndarray):
    """(eps_xc, v_xc) of the unpolarised LDA at each point: Slater exchange
    eps_x = -(3/4)(3 rho/pi)^(1/3), v_x = 4/3 eps_x; Perdew-Zunger correlation in
    rs = (3/(4 pi rho))^(1/3), v_c = eps_c - (rs/3) d eps_c/d rs. Zero where rho <= 0."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    pos = rho > 0.0
    p = rho[pos]
    ex = -0.75 * (3.0 * p / math.pi) ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    rs = (3.0 / (FOUR_PI * p)) ** (1.0 / 3.0)
    ec = np.empty_like(p)
    vc = np.empty_like(p)
    hi = rs >= 1.0
    sq = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    # -(rs/3) d/drs gamma/den = gamma (beta1 sqrt(rs)/6 + beta2 rs/3) / den^2
    vc[hi] = ec[hi] + PZ_GAMMA * (PZ_BETA1 * sq / 6.0 + PZ_BETA2 * rs[hi] / 3.0) / den ** 2
    lo = ~hi
    x = rs[lo]
    lnx = np.log(x)
    ec[lo] = PZ_A * lnx + PZ_B + PZ_C * x * lnx + PZ_D * x
    # d eps/d rs = A/rs + C (ln rs + 1) + D
    vc[lo] = ec[lo] - x / 3.0 * (PZ_A / x + PZ_C * (lnx + 1.0) + PZ_D)
    eps[pos] = ex + ec
    v[pos] = vx + vc
    return eps, v


# ------------------------------------------------------------------------------ occupations
def fermi_occupations(lam: np.ndarray, n_electrons: float, kT: float):
    """Fermi-Dirac occupations f_i = 1 / (1 + exp((lam_i - mu)/kT)) with sum f_i =
    n_electrons / 2 (eq. Fermi_constraint; Sec. 3.4.1), mu by Brent's method. Returns
    (f, mu, S) with the electronic entropy S = -2 sum [f ln f + (1-f) ln(1-f)] (in units of
    k_B; two spins)."""
    from scipy.optimize import brentq
    from scipy.special import expit
    lam = np.asarray(lam, dtype=np.float64)
    target = 0.5 * n_electrons
    if not 0.0 < target < lam.size:
        raise ValueError("need 0 < n_electrons / 2 < number of states")

    def count(mu):
        return float(np.sum(expit(-(lam - mu) / kT))) - target

    lo = lam.min() - 60.0 * kT - 1.0
    hi = lam.max() + 60.0 * kT + 1.0
    mu = brentq(count, lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)
    f = expit(-(lam - mu) / kT)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(f > 0, f * np.log(f), 0.0) + np.where(f < 1, (1 - f) * np.log1p(-f), 0.0)
    return f, mu, float(-2.0 * np.sum(s))


# ------------------------------------------------------------------------------ mixing
class Anderson:
    """Anderson mixing of a grid function x (Sec. 3.4.1): with residuals F_i = g(x_i) - x_i
    and the last m+1 iterates, theta minimises || F_n - sum_j theta_j (F_n - F_{n-j}) ||_W,
    and x_{n+1} = xbar + beta Fbar with xbar = x_n - sum_j theta_j (x_n - x_{n-j}),
    Fbar = F_n - sum_j theta_j (F_n - F_{n-j}). history = m (None: all previous iterates)."""

    def __init__(self, weights: np.ndarray, beta: float, history: int | None = None):
        self.w = np.asarray(weights, dtype=np.float64).ravel()
        self.beta = float(beta)
        self.history = history
        self.xs: list = []
        self.Fs: list = []

    def mix(self, x_in: np.ndarray, x_out: np.ndarray) -> np.ndarray:
        x = np.asarray(x_in, dtype=np.float64).ravel().copy()
        F = np.asarray(x_out, dtype=np.float64).ravel() - x
        self.xs.append(x)
        self.Fs.append(F)
        if self.history is not None and len(self.xs) > self.history + 1:
            self.xs.pop(0)
            self.Fs.pop(0)
        m = len(self.xs) - 1
        if m == 0:
            return (x + self.beta * F).reshape(np.shape(x_in))
        dF = np.stack([F - self.Fs[-1 - j] for j in range(1, m + 1)])  # (m, n)
        dx = np.stack([x - self.xs[-1 - j] for j in range(1, m + 1)])
        A = (dF * self.w) @ dF.T
        b = (dF * self.w) @ F
        theta = np.linalg.solve(A, b)
        xbar = x - theta @ dx
        Fbar = F - theta @ dF
        return (xbar + self.beta * Fbar).reshape(np.shape(x_in))


# ------------------------------------------------------------------------------ SCF
def total_energy(basis: Basis, lam, occ, entropy, kT, rho_out, v_in, v_ext, vh_out, exc_out,
                 e_ion=0.0):
    """Kohn-Sham free energy of the output density (eq. KS_model with the band-energy
    identity): 2 sum f lam - int rho_out (v_in - v_ext) + 1/2 int rho_out V_H[rho_out]
    + int rho_out eps_xc[rho_out] - kT S + E_ion."""
    band = 2.0 * float(np.dot(occ, lam))
    return (band - integral(basis, rho_out, v_in - v_ext) + 0.5 * integral(basis, rho_out, vh_out)
            + integral(basis, rho_out, exc_out) - kT * entropy + e_ion)


def direct_energy(basis: Basis, X, occ, entropy, kT, rho, v_ext, vh, exc, e_ion=0.0):
    """The same functional evaluated term by term: kinetic energy from the coefficients
    (1/2 Lambda diagonal, Sec. 2.2.3), external, Hartree and exchange-correlation energies
    by grid quadrature."""
    X = np.asarray(X, dtype=np.float64)
    ts = 2.0 * float(np.sum(occ * np.sum(basis.half_lambda[:, None] * X * X, axis=0)))
    return (ts + integral(basis, rho, v_ext) + 0.5 * integral(basis, rho, vh)
            + integral(basis, rho, exc) - kT * entropy + e_ion)


def scf(basis: Basis, v_ext: np.ndarray, n_electrons: float, rho0: np.ndarray, n_states: int,
        kT: float = 1e-3, beta: float = 0.3, history: int | None = None, tol: float = 1e-8,
        max_iter: int = 100, e_ion: float = 0.0):
    """SCF loop with potential mixing (Sec. 3.4.1): v_in from the starting density, then
    [lowest n_states eigenpairs of H(v_in) (dense, tiny bases) -> occupations -> density ->
    V_H, LDA -> energy -> Anderson-mixed v_in] until |E_n - E_{n-1}| <= tol."""
    shape = (basis.n_r, basis.n_theta, basis.n_phi)
    v_ext = np.asarray(v_ext, dtype=np.float64).reshape(shape)
    zt = zeta_tables(basis)
    rho0 = np.asarray(rho0, dtype=np.float64).reshape(shape)
    v_in = v_ext + hartree(basis, rho0, zt) + lda_xc(rho0)[1]
    mixer = Anderson(basis.weights(), beta, history)
    energies = []
    out = {}
    for it in range(max_iter):
        H = Hamiltonian(basis, v_in).dense()
        lam_all, vec = np.linalg.eigh(H)
        lam, X = lam_all[:n_states], vec[:, :n_states]
        occ, mu, S = fermi_occupations(lam, n_electrons, kT)
        rho = density(basis, X, occ)
        vh = hartree(basis, rho, zt)
        exc, vxc = lda_xc(rho)
        E = total_energy(basis, lam, occ, S, kT, rho, v_in, v_ext, vh, exc, e_ion)
        energies.append(E)
        out = {"energy": E, "energies": energies, "lam": lam, "occ": occ, "mu": mu,
               "entropy": S, "X": X, "rho": rho, "v_in": v_in, "vh": vh, "exc": exc,
               "iterations": it + 1}
        if it > 0 and abs(energies[-1] - energies[-2]) <= tol:
            out["converged"] = True
            return out
        v_out = v_ext + vh + vxc
        v_in = mixer.mix(v_in, v_out)
    out["converged"] = False
    return out
