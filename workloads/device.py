"""The analytic input functions of `workloads` evaluated with torch, on whatever device the
caller's points live (for grids of millions of points: the 400-atom cluster's grid has
5.5 million nodes and 1600 projector functions).

Input generation only: the same formulas as `erf_cluster_potential` and
`kb_projector_values` (pinned to them by a CPU test), no arithmetic of the spectral method.
"""
from __future__ import annotations

import math

import numpy as np


def erf_cluster_potential_t(xyz, atoms: np.ndarray, Z: float = 4.0, rc: float = 0.8):
    """Sum over atoms of -Z erf(|x-a|/rc)/|x-a| at the points xyz (torch, (n, 3), float64),
    with the series -Z (2/(rc sqrt(pi))) (1 - x^2/3 + x^4/10) for x = r/rc < 1e-3."""
    import torch
    v = torch.zeros(xyz.shape[0], dtype=torch.float64, device=xyz.device)
    c0 = -Z * 2.0 / (rc * math.sqrt(math.pi))
    for a in torch.tensor(np.asarray(atoms, dtype=np.float64), device=xyz.device):
        r = torch.linalg.norm(xyz - a, dim=1)
        x = r / rc
        series = c0 * (1.0 - x * x / 3.0 + x ** 4 / 10.0)
        full = -Z * torch.special.erf(x) / torch.clamp(r, min=1e-300)
        v += torch.where(x < 1e-3, series, full)
    return v


def kb_projector_values_t(xyz, atoms: np.ndarray, rc: float = 1.0, first: int = 0,
                          count: int | None = None):
    """Grid values of the Gaussian s, px, py, pz projectors of atoms[first:first+count]
    (ordered [atom][s, px, py, pz], unit L2(R^3) norm), shape (4 count, n), float64 torch."""
    import torch
    atoms = np.asarray(atoms, dtype=np.float64)
    count = atoms.shape[0] - first if count is None else count
    ns = (math.pi ** 1.5 * rc ** 3) ** -0.5
    npn = (math.pi ** 1.5 * rc ** 5 / 2.0) ** -0.5
    out = torch.empty((4 * count, xyz.shape[0]), dtype=torch.float64, device=xyz.device)
    at = torch.tensor(atoms[first:first + count], device=xyz.device)
    for i in range(count):
        dx = xyz - at[i]
        g = torch.exp(-torch.sum(dx * dx, dim=1) / (2.0 * rc * rc))
        out[4 * i] = ns * g
        out[4 * i + 1] = npn * dx[:, 0] * g
        out[4 * i + 2] = npn * dx[:, 1] * g
        out[4 * i + 3] = npn * dx[:, 2] * g
    return out


def kb_couplings(natoms: int) -> np.ndarray:
    """Couplings of the projectors above (s: +1.0 Ha, p: +0.5 Ha; synthetic values)."""
    return np.tile(np.array([1.0, 0.5, 0.5, 0.5]), natoms)


def gaussian_atom_density_t(xyz, atoms: np.ndarray, Z: float = 4.0, sigma: float = 1.0):
    """SCF starting density of `gaussian_atom_density` (Z electrons per atom in a normalised
    Gaussian of width sigma) at the points xyz (torch, (n, 3), float64)."""
    import torch
    rho = torch.zeros(xyz.shape[0], dtype=torch.float64, device=xyz.device)
    c = Z * (2.0 * math.pi * sigma * sigma) ** -1.5
    for a in torch.tensor(np.asarray(atoms, dtype=np.float64), device=xyz.device):
        d2 = torch.sum((xyz - a) ** 2, dim=1)
        rho += c * torch.exp(-d2 / (2.0 * sigma * sigma))
    return rho
