"""Learned initial density on the GPU (include/cs_learned.h) against the oracle
(oracle/learned_density.py): the atom-centred expansion on the grid, its weighted
least-squares fit, the network's loss and gradients, and Adam training."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import learned_density as LD
from oracle.basis import Basis
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu
SIG = np.array([0.6, 0.9, 1.3, 1.9, 2.8])


def _ctx_basis(R=8.0, lmax=8, N=12, n_r=40, n_t=18, n_p=34):
    torch, cs = need_gpu()
    return torch, cs, cs.cs_basis_init(R, lmax, N, n_r, n_t, n_p, 0, 0), Basis(R, lmax, N, n_r, n_t, n_p)


def test_atom_density_and_fit_match_oracle():
    torch, cs, ctx, b = _ctx_basis()
    a = W.place_atoms(8860, 5, 3.0, 1.5)
    c = W.gaussian_block(8861, 5, len(SIG))
    rho = torch.zeros(b.n_grid, dtype=torch.float64, device="cuda")
    cs.cs_atom_density(ctx, a, SIG, c, rho)
    ref = LD.correction(b.points(), a, SIG, c)
    assert np.max(np.abs(rho.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the fit recovers the planted coefficients, and matches the oracle's fit of a general target
    got = cs.cs_fit_atom_density(ctx, a, SIG, rho, ridge=0.0)
    assert np.max(np.abs(got - c)) <= 1e-7 * np.max(np.abs(c))
    tgt = W.gaussian_atom_density(b.points(), a, Z=4.0, sigma=0.8) - \
        W.gaussian_atom_density(b.points(), a, Z=4.0, sigma=1.0)
    got2 = cs.cs_fit_atom_density(ctx, a, SIG, torch.tensor(tgt, device="cuda"), ridge=1e-10)
    ref2 = LD.fit_coefficients(b.points(), b.weights().ravel(), a, SIG, tgt, ridge=1e-10)
    assert np.max(np.abs(got2 - ref2)) <= 1e-6 * np.max(np.abs(ref2))


def _net(dims, seed=8870):
    params = []
    for i in range(len(dims) - 1):
        params.append(W.gaussian_block(seed + i, dims[i], dims[i + 1]) / math.sqrt(dims[i]))
        params.append(0.1 * W.gaussian(seed + 100 + i, dims[i + 1]))
    flat = np.concatenate([p.ravel(order="F") if p.ndim == 2 else p for p in params])
    return LD.MLP(params), flat.astype(np.float32)


def _unflatten(flat, dims):
    out, o = [], 0
    for i in range(len(dims) - 1):
        k, m = dims[i], dims[i + 1]
        out.append(flat[o:o + k * m].reshape(k, m, order="F"))
        o += k * m
        out.append(flat[o:o + m])
        o += m
    return out


def test_mlp_loss_and_gradients_match_oracle():
    torch, cs = need_gpu()
    dims = [16, 128, 128, 128, 5]
    net, flat = _net(dims)
    n = 300
    X = W.gaussian_block(8880, n, 16)
    T = 0.1 * W.gaussian_block(8881, n, 5)
    m = cs.cs_mlp_create(dims, flat, max_rows=n)
    Xd = torch.tensor(X.T.copy(), dtype=torch.float32, device="cuda")
    Td = torch.tensor(T.T.copy(), dtype=torch.float32, device="cuda")
    Y = cs.cs_mlp_forward(m, Xd).cpu().numpy().T
    net32 = LD.MLP(_unflatten(flat.astype(np.float64), dims))
    assert np.max(np.abs(Y - net32.forward(X))) <= 1e-5 * max(1.0, np.max(np.abs(Y)))
    loss, g = cs.cs_mlp_loss_grad(m, Xd, Td)
    lref, gref = net32.loss_and_grads(X, T)
    assert abs(loss - lref) <= 1e-5 * lref
    gflat = np.concatenate([x.ravel(order="F") if x.ndim == 2 else x for x in gref])
    assert np.max(np.abs(g - gflat)) <= 1e-4 * np.max(np.abs(gflat))


def test_mlp_adam_training_follows_oracle():
    torch, cs = need_gpu()
    dims = [16, 64, 64, 5]
    net, flat = _net(dims, seed=8890)
    n = 200
    X = W.gaussian_block(8891, n, 16)
    T = np.tanh(X[:, :5]) * 0.5 + 0.1 * X[:, 5:10]  # a smooth target the network can fit
    m = cs.cs_mlp_create(dims, flat, max_rows=n)
    Xd = torch.tensor(X.T.copy(), dtype=torch.float32, device="cuda")
    Td = torch.tensor(T.T.copy(), dtype=torch.float32, device="cuda")
    ref = LD.MLP(_unflatten(flat.astype(np.float64), dims))
    opt = LD.Adam(ref.params, lr=3e-3)
    losses_g, losses_o = [], []
    for _ in range(300):
        losses_g.append(cs.cs_mlp_train_step(m, Xd, Td, 3e-3))
        lo, gr = ref.loss_and_grads(X, T)
        losses_o.append(lo)
        opt.step(ref.params, gr)
    assert losses_g[-1] < 0.1 * losses_g[0]
    for k in (0, 50, 299):
        assert abs(losses_g[k] - losses_o[k]) <= 2e-2 * losses_o[k], (k, losses_g[k], losses_o[k])
