"""Pins of the learned-density oracle (oracle/learned_density.py): descriptor invariances, the
radial basis normalisation, exact recovery of planted fit coefficients, the MLP gradients
against finite differences (with a planted mistake), Adam on a convex quadratic, and the
prediction's electron count."""
import math

import numpy as np

import workloads as W
from oracle import learned_density as LD
from oracle.basis import Basis

MU = np.linspace(2.0, 10.0, 16)
SIG = np.array([0.6, 0.9, 1.3, 1.9, 2.8])


def _atoms(seed=8801, n=7):
    return W.place_atoms(seed, n, 4.0, 2.0)


def _rotation(seed=3):
    q, _ = np.linalg.qr(W.gaussian_block(seed, 3, 3))
    return q


def test_descriptors_invariant():
    a = _atoms()
    D = LD.descriptors(a, MU, 0.5)
    Q = _rotation()
    D2 = LD.descriptors(a @ Q.T + np.array([1.0, -2.0, 0.5]), MU, 0.5)
    assert np.max(np.abs(D - D2)) <= 1e-12
    p = np.array([3, 0, 6, 1, 5, 2, 4])
    assert np.max(np.abs(LD.descriptors(a[p], MU, 0.5) - D[p])) <= 1e-12
    # an isolated atom has a zero descriptor
    far = np.vstack([a, [[80.0, 0.0, 0.0]]])
    assert np.max(np.abs(LD.descriptors(far, MU, 0.5)[-1])) <= 1e-300


def test_radial_basis_integrates_to_one():
    """int phi_j d^3x = 1 by radial Gauss-Legendre quadrature of 4 pi r^2 phi_j(r)."""
    x, w = np.polynomial.legendre.leggauss(200)
    r = 20.0 * (1 + x)
    vals = LD.radial_basis(r, SIG) * (4 * math.pi * r[:, None] ** 2) * (20.0 * w)[:, None]
    assert np.max(np.abs(vals.sum(axis=0) - 1.0)) <= 1e-12


def test_fit_recovers_planted_coefficients():
    b = Basis(8.0, 8, 12, 40, 18, 34)
    pts = b.points()
    wts = b.weights().ravel()
    a = _atoms(8802, 4) * 0.6
    c = W.gaussian_block(8803, 4, len(SIG))
    target = LD.correction(pts, a, SIG, c)
    got = LD.fit_coefficients(pts, wts, a, SIG, target, ridge=0.0)
    assert np.max(np.abs(got - c)) <= 1e-7 * np.max(np.abs(c))


def _mlp(seed=8810, dims=(16, 32, 32, 5)):
    params = []
    for i in range(len(dims) - 1):
        params.append(W.gaussian_block(seed + i, dims[i], dims[i + 1]) / math.sqrt(dims[i]))
        params.append(0.1 * W.gaussian(seed + 100 + i, dims[i + 1]))
    return LD.MLP(params)


def test_mlp_gradients_match_finite_differences():
    net = _mlp()
    X = W.gaussian_block(8820, 9, 16)
    T = W.gaussian_block(8821, 9, 5)
    loss, grads = net.loss_and_grads(X, T)
    h = 1e-6
    for k, p in enumerate(net.params):
        flat = p.reshape(-1)
        for idx in (0, flat.size // 2, flat.size - 1):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = net.loss_and_grads(X, T)
            flat[idx] = old - h
            lm, _ = net.loss_and_grads(X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[k].reshape(-1)[idx]) <= 1e-7 * max(1.0, abs(fd)), (k, idx)


def test_planted_wrong_tanh_derivative_breaks_gradient_check():
    net = _mlp()
    X = W.gaussian_block(8822, 9, 16)
    T = W.gaussian_block(8823, 9, 5)
    Y, acts = net.forward(X, keep=True)
    # planted: backward through tanh with (1 - h) instead of (1 - h^2)
    d = 2.0 * (Y - T) / Y.size
    d = d @ net.params[4].T * (1.0 - acts[2])
    g1_bad = acts[1].T @ d
    _, grads = net.loss_and_grads(X, T)
    assert np.max(np.abs(g1_bad - grads[2])) > 1e-3 * np.max(np.abs(grads[2]))


def test_adam_minimises_quadratic():
    rng_target = W.gaussian(8830, 6)
    p = [np.zeros(6)]
    opt = LD.Adam(p, lr=0.05)
    for _ in range(3000):
        opt.step(p, [2.0 * (p[0] - rng_target)])
    assert np.max(np.abs(p[0] - rng_target)) <= 1e-4


def test_predicted_density_has_the_electron_count():
    b = Basis(8.0, 6, 10, 30, 14, 28)
    pts = b.points()
    wts = b.weights().ravel()
    a = _atoms(8840, 3) * 0.5
    rho0 = W.gaussian_atom_density(pts, a, Z=2.0, sigma=1.0)
    c = 0.05 * W.gaussian_block(8841, 3, len(SIG))
    rho = LD.predicted_density(pts, wts, a, SIG, c, rho0, 6.0)
    assert abs(np.sum(wts * rho) - 6.0) <= 1e-10
