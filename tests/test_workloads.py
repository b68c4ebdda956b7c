"""Seeded input generators: SplitMix64 against its published test vector, Box-Muller
moments, atom placement constraints."""
import numpy as np

import workloads as W


def test_splitmix64_published_vector():
    # first five outputs for seed 1234567 of the reference SplitMix64 (Steele et al. 2014)
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert list(map(int, W.splitmix64(1234567, 5))) == ref
    # counter-based: an offset window equals the tail of a longer draw
    assert np.array_equal(W.splitmix64(42, 10)[4:], W.splitmix64(42, 6, offset=4))


def test_gaussian_moments():
    g = W.gaussian(5, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1.0) < 0.01


def test_gaussian_block_is_column_major():
    g = W.gaussian(3, 12)
    B = W.gaussian_block(3, 4, 3)
    assert np.array_equal(B[:, 1], g[4:8])


def test_atom_placement():
    w = W.erf_cluster_32()
    a = w.atoms()
    assert a.shape == (32, 3)
    assert np.all(np.linalg.norm(a, axis=1) <= 8.0 + 1e-12)
    dd = np.linalg.norm(a[:, None, :] - a[None, :, :], axis=2) + np.eye(32) * 1e9
    assert dd.min() >= 3.5
    assert np.array_equal(a, w.atoms())  # seeded


def test_erf_atom_limit():
    # -Z erf(r/rc)/r -> -2Z/(rc sqrt(pi)) at r = 0 and continuity across the series switch
    v0 = W.erf_atom_radial(np.array([0.0]), 4.0, 0.8)[0]
    assert abs(v0 + 8.0 / (0.8 * np.sqrt(np.pi))) < 1e-15
    r = np.array([0.8e-3 * (1 - 1e-9), 0.8e-3 * (1 + 1e-9)])
    v = W.erf_atom_radial(r, 4.0, 0.8)
    assert abs(v[0] - v[1]) < 1e-12


def test_kb_projector_norm():
    # analytic normalisation: integrate |p|^2 on a fine Cartesian grid
    h = 0.08
    ax = np.arange(-6, 6 + h / 2, h)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    p, hh = W.kb_projector_values(xyz, np.zeros((1, 3)), rc=1.0)
    norms = (p ** 2).sum(axis=1) * h ** 3
    assert np.allclose(norms, 1.0, atol=1e-6)
    assert list(hh) == [1.0, 0.5, 0.5, 0.5]


def test_torch_generators_equal_numpy_ones():
    """The torch evaluations used for large grids reproduce the numpy input functions."""
    import torch

    from workloads.device import (erf_cluster_potential_t, gaussian_atom_density_t, kb_couplings,
                                  kb_projector_values_t)
    u = W.uniform(99, 3 * 500).reshape(500, 3) * 12.0 - 6.0
    u[0] = [0.0, 0.0, 0.0]          # on an atom: series branch
    atoms = W.place_atoms(98, 5, 4.0, 2.0)
    u[1] = atoms[2] + 1e-5          # near an atom
    v_np = W.erf_cluster_potential(u, atoms, 4.0, 0.8)
    v_t = erf_cluster_potential_t(torch.tensor(u), atoms, 4.0, 0.8).numpy()
    assert np.max(np.abs(v_np - v_t)) <= 1e-13 * np.max(np.abs(v_np))
    p_np, h_np = W.kb_projector_values(u, atoms, rc=1.0)
    p_t = kb_projector_values_t(torch.tensor(u), atoms, rc=1.0, first=1, count=3).numpy()
    assert np.max(np.abs(p_np[4:16] - p_t)) <= 1e-14
    assert np.array_equal(h_np, kb_couplings(5))
    r_np = W.gaussian_atom_density(u, atoms, 4.0, 1.0)
    r_t = gaussian_atom_density_t(torch.tensor(u), atoms, 4.0, 1.0).numpy()
    assert np.max(np.abs(r_np - r_t)) <= 1e-14 * np.max(r_np)
