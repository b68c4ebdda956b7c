"""LOBPCG on the GPU (cs_lobpcg) against the dense eigenvalues and the oracle's LOBPCG on the
same seeded block, with and without the Teter-Payne-Allan preconditioner, on a small block
and on a block whose Rayleigh-Ritz matrices exceed the eigensolver's shared-memory form."""
import numpy as np
import pytest

import workloads as W
from oracle import lobpcg as OL
from oracle.basis import basis_for
from oracle.hamiltonian import Hamiltonian
from tests.gpu_common import make_ctx, need_gpu

pytestmark = pytest.mark.gpu


def _case(lmax, nmax, n_r, n_t, n_p, n_s, seed):
    w = W.small_cluster(lmax=lmax, nmax=nmax, n_r=n_r, n_theta=n_t, n_phi=n_p, n_s=n_s,
                        seed=seed)
    b = basis_for(w)
    return w, b, Hamiltonian(b, w.potential_at(b.points()))


@pytest.mark.parametrize("pre", [True, False])
def test_lobpcg_matches_dense_and_oracle(pre):
    torch, cs = need_gpu()
    w, b, H = _case(5, 8, 16, 12, 24, 12, 7301)
    lam = np.linalg.eigvalsh(H.dense())
    X0 = W.gaussian_block(7302, b.d, 12)
    ref = OL.lobpcg(H.apply, X0, 10, 2 * b.half_lambda if pre else None, tol=1e-9, max_iter=300)
    ctx = make_ctx(w)
    X = torch.zeros((12, b.d + 5), dtype=torch.float64, device="cuda")
    X[:, :b.d] = torch.tensor(X0.T.copy(), device="cuda")
    theta = torch.empty(12, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    it, rs = cs.cs_lobpcg(ctx, X, 10, theta, resid, tol=1e-9, max_iter=300, precondition=pre)
    th = theta.cpu().numpy()
    assert np.max(resid.cpu().numpy()[:10]) <= 1e-9
    assert np.max(np.abs(th[:10] - lam[:10])) <= 1e-10
    assert np.max(np.abs(th[:10] - ref[0][:10])) <= 1e-10
    Xh = X[:, :b.d].cpu().numpy().T
    assert np.max(np.abs(Xh.T @ Xh - np.eye(12))) <= 1e-11
    # the same algorithm on the same block: iteration counts agree closely
    assert abs(it - ref[3]) <= 3


def test_lobpcg_large_block():
    """48 states (Rayleigh-Ritz matrices up to 144 x 144)."""
    torch, cs = need_gpu()
    w, b, H = _case(6, 10, 20, 14, 28, 48, 7311)
    lam = np.linalg.eigvalsh(H.dense())
    ctx = make_ctx(w)
    X = torch.tensor(W.gaussian_block(7312, b.d, 48).T.copy(), device="cuda")
    theta = torch.empty(48, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    it, rs = cs.cs_lobpcg(ctx, X, 40, theta, resid, tol=1e-8, max_iter=400)
    assert np.max(np.abs(theta.cpu().numpy()[:40] - lam[:40])) <= 1e-9
    assert np.max(resid.cpu().numpy()[:40]) <= 1e-8


def test_lobpcg_on_a_larger_basis_matches_chfsi():
    """d = 4056, 40 states: the narrow Gram products of an iteration split d into more row
    chunks than the widest one, so their partial sums need more room (the workspace is sized
    for every shape); eigenvalues equal those of a tightly converged FP64 ChFSI."""
    torch, cs = need_gpu()
    w = W.small_cluster(lmax=12, nmax=24, n_r=48, n_theta=26, n_phi=50, n_s=40, seed=7321,
                        R=10.0, natoms=4)
    ctx = make_ctx(w)
    d = ctx.d
    X0 = torch.tensor(W.gaussian_block(7322, d, 40).T.copy(), device="cuda")
    theta = torch.empty(40, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    X = X0.clone()
    it, rs = cs.cs_lobpcg(ctx, X, 32, theta, resid, tol=1e-8, max_iter=300)
    assert rs == 0
    th_lb = theta.cpu().numpy()[:32].copy()
    v0 = torch.tensor(W.gaussian(7323, d), device="cuda")
    X = X0.clone()
    cs.cs_chfsi(ctx, X, 32, 16, v0, theta, resid, tol=1e-9, max_iter=200)
    assert np.max(np.abs(th_lb - theta.cpu().numpy()[:32])) <= 1e-9
