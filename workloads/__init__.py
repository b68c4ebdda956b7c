"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the spectral method itself: no basis, no
quadrature, no transform, no Hamiltonian. It only provides
  * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014) as a counter-based stream, uniform doubles from it
    and Box-Muller Gaussians;
  * seeded atom placement (random sequential addition with a minimum separation);
  * analytic potentials and projector functions evaluated at points the caller
    supplies (each side evaluates them on its own quadrature grid):
      - 3-D harmonic oscillator 1/2 w^2 |x-c|^2,
      - a sum of local pseudo-atoms  -Z erf(|x-a|/rc)/|x-a|  (the local
        pseudopotential is a superposition of radial atom terms, Sec. 2.3.2),
      - Gaussian s and p Kleinman-Bylander projector functions (the non-local
        term is a sum of rank-one atom-centred projectors, Sec. 2.3.2);
  * the workload descriptions (sizes, seeds) of the synthetic clusters.

Both the CPU oracle and the CUDA product read their inputs from here; neither
imports the other.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of the SplitMix64 stream started at state `seed`.

    Output i is mix(seed + (i+1)*gamma) (mod 2^64), which is what the
    sequential generator returns as its i-th value.
    """
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of each SplitMix64 output."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * np.pi * u2)
    out[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return out[:n]


def gaussian_block(seed: int, d: int, n_s: int) -> np.ndarray:
    """d x n_s block of N(0,1) values, filled in column-major order."""
    return gaussian(seed, d * n_s).reshape(n_s, d).T.copy()  # column s = values s*d .. s*d+d-1


def place_atoms(seed: int, natoms: int, r_place: float, min_sep: float,
                max_tries: int = 2_000_000) -> np.ndarray:
    """Random sequential addition of `natoms` points uniformly in the ball |x| <= r_place.

    A candidate uses three consecutive uniforms (u, v, w): radius r_place*u^(1/3),
    cos(theta) = 2v - 1, phi = 2 pi w. It is kept if it is at least `min_sep`
    from every atom kept before it.
    """
    atoms = np.zeros((natoms, 3))
    count = 0
    chunk = 3 * 4096
    offset = 0
    tries = 0
    while count < natoms:
        u = uniform(seed, chunk, offset)
        offset += chunk
        for c in range(chunk // 3):
            tries += 1
            if tries > max_tries:
                raise RuntimeError("atom placement did not finish; packing too dense")
            rr = r_place * u[3 * c] ** (1.0 / 3.0)
            ct = 2.0 * u[3 * c + 1] - 1.0
            st = math.sqrt(max(0.0, 1.0 - ct * ct))
            ph = 2.0 * math.pi * u[3 * c + 2]
            p = np.array([rr * st * math.cos(ph), rr * st * math.sin(ph), rr * ct])
            if count == 0 or np.min(np.sum((atoms[:count] - p) ** 2, axis=1)) >= min_sep * min_sep:
                atoms[count] = p
                count += 1
                if count == natoms:
                    break
    return atoms


# --------------------------------------------------------------------------------------
# analytic functions evaluated at caller-supplied points (xyz: (n, 3))
# --------------------------------------------------------------------------------------

def ho_potential(xyz: np.ndarray, omega: float = 1.0, center=(0.3, -0.2, 0.1)) -> np.ndarray:
    """1/2 omega^2 |x - c|^2."""
    d = xyz - np.asarray(center, dtype=np.float64)[None, :]
    return 0.5 * omega * omega * np.sum(d * d, axis=1)


def _erf(x: np.ndarray) -> np.ndarray:
    from scipy.special import erf  # scipy is present on both machines
    return erf(x)


def erf_atom_radial(r: np.ndarray, Z: float = 4.0, rc: float = 0.8) -> np.ndarray:
    """-Z erf(r/rc)/r, with its series near r = 0 (limit -2Z/(rc sqrt(pi)))."""
    r = np.asarray(r, dtype=np.float64)
    x = r / rc
    out = np.empty_like(r)
    small = x < 1e-3
    xs = x[small]
    out[small] = -Z * (2.0 / (rc * math.sqrt(math.pi))) * (1.0 - xs * xs / 3.0 + xs ** 4 / 10.0)
    rl = r[~small]
    out[~small] = -Z * _erf(rl / rc) / rl
    return out


def erf_cluster_potential(xyz: np.ndarray, atoms: np.ndarray, Z: float = 4.0,
                          rc: float = 0.8) -> np.ndarray:
    """Sum over atoms of -Z erf(|x-a|/rc)/|x-a| (local pseudo-atoms)."""
    v = np.zeros(xyz.shape[0])
    for a in atoms:
        r = np.sqrt(np.sum((xyz - a[None, :]) ** 2, axis=1))
        v += erf_atom_radial(r, Z, rc)
    return v


def kb_projector_values(xyz: np.ndarray, atoms: np.ndarray, rc: float = 1.0):
    """Grid values of Gaussian s and p projectors on each atom, unit L2(R^3) norm.

    Returns (p, h): p has shape (4*natoms, n) ordered [atom][s, px, py, pz];
    h are the couplings (s: +1.0 Ha, p: +0.5 Ha; synthetic values).
    """
    n = xyz.shape[0]
    na = atoms.shape[0]
    p = np.empty((4 * na, n))
    ns = (math.pi ** 1.5 * rc ** 3) ** -0.5
    npn = (math.pi ** 1.5 * rc ** 5 / 2.0) ** -0.5
    for i, a in enumerate(atoms):
        dx = xyz - a[None, :]
        g = np.exp(-np.sum(dx * dx, axis=1) / (2.0 * rc * rc))
        p[4 * i] = ns * g
        p[4 * i + 1] = npn * dx[:, 0] * g
        p[4 * i + 2] = npn * dx[:, 1] * g
        p[4 * i + 3] = npn * dx[:, 2] * g
    h = np.tile(np.array([1.0, 0.5, 0.5, 0.5]), na)
    return p, h


def gaussian_atom_density(xyz: np.ndarray, atoms: np.ndarray, Z: float = 4.0,
                          sigma: float = 1.0) -> np.ndarray:
    """SCF starting density: Z electrons per atom in a normalised Gaussian of width sigma,
    Z (2 pi sigma^2)^(-3/2) exp(-|x-a|^2 / (2 sigma^2)), summed over atoms (a synthetic
    superposition of atomic densities)."""
    rho = np.zeros(xyz.shape[0])
    c = Z * (2.0 * math.pi * sigma * sigma) ** -1.5
    for a in atoms:
        d2 = np.sum((xyz - a[None, :]) ** 2, axis=1)
        rho += c * np.exp(-d2 / (2.0 * sigma * sigma))
    return rho


# --------------------------------------------------------------------------------------
# workload descriptions
# --------------------------------------------------------------------------------------

@dataclass
class Workload:
    """One synthetic cluster problem: basis, quadrature, potential and block sizes."""
    name: str
    R: float
    lmax: int
    nmax: int              # radial functions per l
    n_r: int
    n_theta: int
    n_phi: int
    radial_rule: str       # "gauss_legendre" or "gauss_jacobi_r2"
    n_s: int               # states in the block
    degree: int            # Chebyshev degree
    potential: str         # "ho", "erf_cluster", "zero", "const"
    natoms: int = 0
    atom_seed: int = 0
    r_place: float = 0.0
    min_sep: float = 3.5
    x_seed: int = 0
    n_want: int = 0
    kb: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return self.lmax + 1

    @property
    def d(self) -> int:
        return self.L * self.L * self.nmax

    @property
    def n_grid(self) -> int:
        return self.n_r * self.n_theta * self.n_phi

    def atoms(self) -> np.ndarray:
        if self.natoms == 0:
            return np.zeros((0, 3))
        return place_atoms(self.atom_seed, self.natoms, self.r_place, self.min_sep)

    def potential_at(self, xyz: np.ndarray) -> np.ndarray:
        if self.potential == "ho":
            return ho_potential(xyz, self.extra.get("omega", 1.0),
                                self.extra.get("center", (0.3, -0.2, 0.1)))
        if self.potential == "erf_cluster":
            return erf_cluster_potential(xyz, self.atoms(), self.extra.get("Z", 4.0),
                                         self.extra.get("rc", 0.8))
        if self.potential == "zero":
            return np.zeros(xyz.shape[0])
        if self.potential == "const":
            return np.full(xyz.shape[0], float(self.extra.get("v0", 0.0)))
        raise ValueError(self.potential)

    def x_block(self, n_s: int | None = None) -> np.ndarray:
        return gaussian_block(self.x_seed, self.d, self.n_s if n_s is None else n_s)


def harmonic_oscillator_ball() -> Workload:
    """H = -1/2 Lap + 1/2 |x-c|^2, c = (0.3,-0.2,0.1), R = 8, lmax 10, 16 radial functions,
    32 x 22 x 42 Gauss-Legendre grid; 16-state block (10 wanted), degree 12."""
    return Workload("ho_ball_l10_n16", R=8.0, lmax=10, nmax=16, n_r=32, n_theta=22, n_phi=42,
                    radial_rule="gauss_legendre", n_s=16, degree=12, potential="ho",
                    x_seed=1001, n_want=10, extra={"omega": 1.0, "center": (0.3, -0.2, 0.1)})


def erf_cluster_32() -> Workload:
    """32 erf pseudo-atoms (Z=4, rc=0.8) in r <= 8, min separation 3.5, ball R = 14,
    lmax 30, 48 radial functions (d = 46128), 96 x 60 x 120 grid, 80 states, degree 16."""
    return Workload("erf32_l30_n48", R=14.0, lmax=30, nmax=48, n_r=96, n_theta=60, n_phi=120,
                    radial_rule="gauss_legendre", n_s=80, degree=16, potential="erf_cluster",
                    natoms=32, atom_seed=2001, r_place=8.0, min_sep=3.5, x_seed=2002, n_want=64,
                    extra={"Z": 4.0, "rc": 0.8})


def erf_cluster_400_kb() -> Workload:
    """400 erf pseudo-atoms with Gaussian s,p projectors (rc = 1) in r <= 18, ball R = 26,
    lmax 60, 96 radial functions (d = 357216), 192 x 120 x 240 grid, 880 states in chunks
    of 128, degree 20."""
    return Workload("erf400kb_l60_n96", R=26.0, lmax=60, nmax=96, n_r=192, n_theta=120,
                    n_phi=240, radial_rule="gauss_legendre", n_s=880, degree=20,
                    potential="erf_cluster", natoms=400, atom_seed=3001, r_place=18.0,
                    min_sep=3.5, x_seed=3002, n_want=800, kb=True,
                    extra={"Z": 4.0, "rc": 0.8, "kb_rc": 1.0, "chunk": 128})


def batched_clusters(count: int = 96, seed0: int = 4000) -> list:
    """`count` clusters of 4-48 erf pseudo-atoms; R, lmax and N grow with the cluster size."""
    out = []
    for i in range(count):
        u = uniform(seed0 + i, 4)
        natoms = 4 + int(u[0] * 45)  # 4 .. 48
        r_place = 1.75 * (natoms / 0.15) ** (1.0 / 3.0) - 1.75  # packing fraction 0.15
        rmin = max(8.0, r_place + 6.0)
        R = rmin + (16.0 - rmin) * u[1] if rmin < 16.0 else 16.0
        r_place = min(r_place, R - 6.0)
        lmax = int(round(12 + 20 * (R - 8.0) / 8.0))
        nmax = int(round(24 + 32 * (R - 8.0) / 8.0))
        n_s = min(128, int(math.ceil(2.4 * natoms)))
        out.append(Workload(f"batch{i}", R=R, lmax=lmax, nmax=nmax, n_r=2 * nmax,
                            n_theta=2 * lmax, n_phi=4 * lmax, radial_rule="gauss_legendre",
                            n_s=n_s, degree=16, potential="erf_cluster", natoms=natoms,
                            atom_seed=seed0 + i, r_place=r_place, min_sep=3.5,
                            x_seed=4100 + i, n_want=2 * natoms,
                            extra={"Z": 4.0, "rc": 0.8}))
    return out


def small_cluster(lmax=6, nmax=8, n_r=20, n_theta=14, n_phi=28, R=8.0, n_s=12,
                  natoms=3, seed=7001, potential="erf_cluster") -> Workload:
    """A small erf cluster for tests that compare against dense matrices."""
    name = f"small_l{lmax}_n{nmax}_r{n_r}x{n_theta}x{n_phi}_R{R:g}_s{n_s}_a{natoms}_{seed}_{potential}"
    return Workload(name, R=R, lmax=lmax, nmax=nmax, n_r=n_r,
                    n_theta=n_theta, n_phi=n_phi, radial_rule="gauss_legendre", n_s=n_s,
                    degree=8, potential=potential, natoms=natoms, atom_seed=seed,
                    r_place=3.0, min_sep=2.0, x_seed=seed + 1, n_want=n_s // 2,
                    extra={"Z": 4.0, "rc": 0.8})
