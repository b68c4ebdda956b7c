"""GPU parity of the Chebyshev filter, Cholesky-QR, Rayleigh-Ritz, the Lanczos bound, the
projector pair and the ChFSI loop against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen
from tests.gpu_common import make_ctx, need_gpu, oracle_H, register, rel_errors, to_dev, to_host

pytestmark = pytest.mark.gpu

SMALL = W.small_cluster(lmax=6, nmax=8, n_r=20, n_theta=14, n_phi=28, n_s=13)
HO = W.harmonic_oscillator_ball()
register(SMALL)
register(HO)


def _bounds(Hh):
    lam = np.linalg.eigvalsh(Hh.dense())
    return float(lam[24]), float(lam[-1]) + 1.0, float(lam[0]), lam


@pytest.mark.parametrize("degree", [1, 2, 9])
def test_cheb_filter_fp64_matches_oracle(degree):
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    a, b, a0, _ = _bounds(Hh)
    X = w.x_block()
    ref = eigen.cheb_filter(Hh.apply, X, degree, a, b, a0)
    Xd = to_dev(X, ld=ctx.d + 5)
    cs.cs_cheb_filter(ctx, Xd, degree, a, b, a0, cs.CS_FP64)
    torch.cuda.synchronize()
    fro, col = rel_errors(to_host(Xd, ctx.d), ref)
    assert fro <= 1e-11 and col <= 1e-11, (fro, col)


def test_cheb_filter_fp32_error():
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    a, b, a0, _ = _bounds(Hh)
    X = w.x_block()
    ref = eigen.cheb_filter(Hh.apply, X, 8, a, b, a0)
    Xd = to_dev(X, dtype=torch.float32)
    cs.cs_cheb_filter(ctx, Xd, 8, a, b, a0, cs.CS_FP32)
    torch.cuda.synchronize()
    fro, _ = rel_errors(to_host(Xd, ctx.d), ref)
    assert fro <= 1e-4, fro


def test_cheb_filter_rejects_bad_bounds():
    torch, cs = need_gpu()
    ctx = make_ctx(SMALL)
    Xd = to_dev(SMALL.x_block())
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_cheb_filter(ctx, Xd, 4, 5.0, 1.0, 0.0)


def test_cholqr_matches_oracle():
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((ctx.d, 13)) @ np.diag(np.logspace(0, 4, 13))
    ref = eigen.cholqr(X)
    Xd = to_dev(X, ld=ctx.d + 1)
    cs.cs_cholqr(ctx, Xd)
    torch.cuda.synchronize()
    got = to_host(Xd, ctx.d)
    assert np.max(np.abs(got.T @ got - np.eye(13))) < 1e-13
    assert np.max(np.abs(got - ref)) < 1e-10


def test_cholqr_rank_deficient_reports_breakdown():
    torch, cs = need_gpu()
    ctx = make_ctx(SMALL)
    X = np.ones((ctx.d, 4))
    with pytest.raises(cs.CsError, match="CS_ERR_CHOLESKY"):
        cs.cs_cholqr(ctx, to_dev(X))


def test_rayleigh_ritz_matches_oracle():
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    X = eigen.cholqr(w.x_block())
    th_ref, X_ref, HX_ref, res_ref = eigen.rayleigh_ritz(Hh.apply, X)
    Xd = to_dev(X)
    theta = torch.empty(13, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    HXo = torch.empty_like(Xd)
    cs.cs_rayleigh_ritz(ctx, Xd, theta, resid, HXo)
    torch.cuda.synchronize()
    assert np.max(np.abs(theta.cpu().numpy() - th_ref)) < 1e-11 * np.abs(th_ref).max()
    assert np.max(np.abs(resid.cpu().numpy() - res_ref)) < 1e-10 * np.abs(res_ref).max()
    # Ritz vectors agree up to sign (eigenvalues of a random projection are simple)
    got = to_host(Xd, ctx.d)
    sgn = np.sign(np.sum(got * X_ref, axis=0))
    assert np.max(np.abs(got * sgn - X_ref)) < 1e-9


def test_lanczos_bound_matches_oracle():
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    v0 = W.gaussian(31, ctx.d)
    b_ref, t_ref = eigen.lanczos_bound(Hh.apply, v0, 10)
    b, tmin = cs.cs_lanczos_bound(ctx, torch.tensor(v0, device="cuda"), 10)
    assert abs(b - b_ref) < 1e-9 * abs(b_ref) and abs(tmin - t_ref) < 1e-9 * abs(b_ref)
    lam = np.linalg.eigvalsh(Hh.dense())
    assert b >= lam[-1]


def test_chfsi_small_cluster_vs_dense():
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    lam = np.linalg.eigvalsh(oracle_H(w.name).dense())
    Xd = to_dev(w.x_block())
    theta = torch.empty(13, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    v0 = torch.tensor(W.gaussian(9, ctx.d), device="cuda")
    it = cs.cs_chfsi(ctx, Xd, 6, 10, v0, theta, resid, tol=1e-10, max_iter=100)
    th = theta.cpu().numpy()
    assert it >= 1
    assert np.max(resid.cpu().numpy()[:6]) <= 1e-10
    assert np.max(np.abs(th[:6] - lam[:6])) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_chfsi_harmonic_oscillator(precision):
    """lmax 10, 16 radial functions, R = 8: the ten lowest levels 1.5, 2.5 x3, 3.5 x6 Ha."""
    torch, cs = need_gpu()
    w = HO
    ctx = make_ctx(w)
    Xd = to_dev(w.x_block())
    theta = torch.empty(w.n_s, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    v0 = torch.tensor(W.gaussian(99, ctx.d), device="cuda")
    prec = cs.CS_FP64 if precision == "fp64" else cs.CS_FP32
    tol = 1e-8 if precision == "fp64" else 1e-5
    cs.cs_chfsi(ctx, Xd, w.n_want, w.degree, v0, theta, resid, tol=tol, max_iter=60,
                precision=prec)
    th = theta.cpu().numpy()[:10]
    lev = np.loadtxt(__file__.replace("test_gpu_eigen.py", "golden/ho_levels.txt"))
    assert np.max(np.abs(th - lev)) < 1e-6
    if precision == "fp64":
        # against the oracle's dense eigenvalues (1e-9 Ha bar)
        lam = np.linalg.eigvalsh(oracle_H(w.name).dense())
        assert np.max(np.abs(th - lam[:10])) < 1e-9


def test_projector_pair_matches_oracle():
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    from oracle.hamiltonian import Hamiltonian
    b = oracle_H(w.name).basis
    atoms = np.array([[0.0, 0.0, 0.0], [1.0, -0.5, 0.7]])
    v = w.potential_at(b.points())
    pg_o, h = W.kb_projector_values(b.points(), atoms, rc=1.0)
    Hkb = Hamiltonian(b, v, pg_o, h)
    X = w.x_block()
    ref = Hkb.apply(X)
    # the library forward-transforms the projectors sampled on its own grid
    pg = W.kb_projector_values(cs.grid_points(ctx), atoms, rc=1.0)[0]
    pg_d = torch.tensor(pg.reshape(-1, ctx.n_r, ctx.n_theta, ctx.n_phi), device="cuda")
    pcoef = torch.empty((pg.shape[0], ctx.d), dtype=torch.float64, device="cuda")
    cs.cs_forward_transform(ctx, pg_d, pcoef)
    cs.cs_set_projectors(ctx, pcoef, h)
    Xd = to_dev(X)
    HXd = torch.empty_like(Xd)
    cs.cs_apply_H(ctx, Xd, HXd, cs.CS_FP64)
    torch.cuda.synchronize()
    fro, col = rel_errors(to_host(HXd, ctx.d), ref)
    assert fro <= 1e-11 and col <= 1e-11, (fro, col)
