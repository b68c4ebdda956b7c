"""GPU parity of the residual form of the Chebyshev filter (cs_cheb_filter_ritz,
cs_chfsi_step_ritz) against the oracle's plain filter, through the C ABI.

For a block X, any diagonal Theta and R = H X - X Theta, the scaled filter p_m(H) X equals
X s_m(Theta) + D_m with D run through the same recurrence from D_0 = 0, D_1 = (sigma_1/e) R
and the source R s_i(Theta) at every step (Sec. 3.2.1's filter, regrouped). The oracle never
uses that regrouping: every expected value here is its plain recurrence."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen
from tests.gpu_common import make_ctx, need_gpu, oracle_H, register, rel_errors, to_dev, to_host

pytestmark = pytest.mark.gpu

SMALL = W.small_cluster(lmax=6, nmax=8, n_r=20, n_theta=14, n_phi=28, n_s=13)
register(SMALL)


def _bounds(Hh):
    lam = np.linalg.eigvalsh(Hh.dense())
    return float(lam[24]), float(lam[-1]) + 1.0, float(lam[0]), lam


@pytest.mark.parametrize("precision", ["fp64", "df64"])
@pytest.mark.parametrize("degree", [1, 2, 9])
def test_cheb_filter_ritz_matches_oracle_for_any_theta(degree, precision):
    """Arbitrary block and arbitrary theta (not Ritz values): the regrouping is an identity,
    so the FP64 and double-float results hold the 1e-11 bar against the plain recurrence."""
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    a, b, a0, _ = _bounds(Hh)
    X = w.x_block()
    HX = Hh.apply(X)
    theta = np.linspace(a0, b, X.shape[1])[::-1].copy()  # unordered values across the spectrum
    ref = eigen.cheb_filter(Hh.apply, X, degree, a, b, a0)
    Xd = to_dev(X, ld=ctx.d + 5)
    HXd = to_dev(HX, ld=ctx.d + 2)
    thd = torch.tensor(theta, device="cuda")
    cs.cs_cheb_filter_ritz(ctx, Xd, HXd, thd, degree, a, b, a0,
                           cs.CS_FP64 if precision == "fp64" else cs.CS_DF64)
    torch.cuda.synchronize()
    fro, col = rel_errors(to_host(Xd, ctx.d), ref)
    assert fro <= 1e-11 and col <= 1e-11, (fro, col)
    # HX is read only
    assert np.array_equal(to_host(HXd, ctx.d), HX)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_cheb_filter_ritz_error_follows_the_residual(precision):
    """Near-converged Ritz vectors (exact eigenvectors plus a 1e-6 perturbation, then the
    oracle's Rayleigh-Ritz): the residual form's error is the reduced precision's rounding
    times about ||R|| / ||X||, so it sits far below the plain form's error for the same
    block."""
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    a, b, a0, lam = _bounds(Hh)
    _, V = np.linalg.eigh(Hh.dense())
    rng = np.random.default_rng(5)
    X = V[:, :13] + 1e-6 * rng.standard_normal((ctx.d, 13))
    th, Xr, HXr, res = eigen.rayleigh_ritz(Hh.apply, eigen.cholqr(X))
    a = float(th[-1]) + 0.5 * float(lam[13] - th[-1])
    a0 = float(th[0])
    degree = 8
    ref = eigen.cheb_filter(Hh.apply, Xr, degree, a, b, a0)
    prec = cs.CS_FP32 if precision == "fp32" else cs.CS_MIXED_BF16
    Xd = to_dev(Xr)
    cs.cs_cheb_filter_ritz(ctx, Xd, to_dev(HXr), torch.tensor(th, device="cuda"), degree, a, b,
                           a0, prec)
    Xp = to_dev(Xr, dtype=torch.float32)
    cs.cs_cheb_filter(ctx, Xp, degree, a, b, a0, prec)
    torch.cuda.synchronize()
    fro_r, col_r = rel_errors(to_host(Xd, ctx.d), ref)
    fro_p, _ = rel_errors(to_host(Xp, ctx.d), ref)
    print(f"{precision}: residual form {fro_r:.2e} (column {col_r:.2e}), plain {fro_p:.2e}, "
          f"max residual {np.max(res):.2e}")
    # measured on a GB300: FP32 2.6e-12 against 4.3e-7 plain, mixed 9.2e-11 against 1.3e-5,
    # with the block's largest residual 1.4e-4
    assert fro_r <= 1e-4 * fro_p, (fro_r, fro_p)
    assert fro_r <= {"fp32": 8e-12, "mixed": 3e-10}[precision], fro_r


def test_chfsi_step_ritz_matches_oracle_iteration():
    """One ChFSI iteration with the residual-form filter in FP64 (filter, Cholesky-QR twice,
    Rayleigh-Ritz) against the oracle's plain iteration from the same Ritz block: the same
    Ritz values and residuals, and the outgoing H X equals H applied to the new Ritz vectors."""
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    a, b, a0, lam = _bounds(Hh)
    th0, X0, HX0, _ = eigen.rayleigh_ritz(Hh.apply, eigen.cholqr(w.x_block()))
    a, a0 = float(th0[-1]), float(th0[0])
    Y = eigen.cholqr(eigen.cholqr(eigen.cheb_filter(Hh.apply, X0, 6, a, b, a0)))
    th_ref, X_ref, _, res_ref = eigen.rayleigh_ritz(Hh.apply, Y)
    Xd = to_dev(X0)
    HXd = to_dev(HX0)
    theta = torch.tensor(th0, device="cuda")
    resid = torch.empty_like(theta)
    cs.cs_chfsi_step_ritz(ctx, Xd, HXd, 6, a, b, a0, theta, resid, cs.CS_FP64)
    torch.cuda.synchronize()
    th = theta.cpu().numpy()
    assert np.max(np.abs(th - th_ref)) < 1e-11 * np.abs(th_ref).max()
    assert np.max(np.abs(resid.cpu().numpy() - res_ref)) < 1e-9 * np.abs(res_ref).max()
    Xg = to_host(Xd, ctx.d)
    fro, col = rel_errors(to_host(HXd, ctx.d), Hh.apply(Xg))
    assert fro <= 1e-11 and col <= 1e-11, (fro, col)


def test_cheb_filter_ritz_rejects_bad_arguments():
    torch, cs = need_gpu()
    ctx = make_ctx(SMALL)
    Xd = to_dev(SMALL.x_block())
    th = torch.zeros(13, dtype=torch.float64, device="cuda")
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_cheb_filter_ritz(ctx, Xd, Xd.clone(), th, 65, 1.0, 5.0, 0.0)
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_cheb_filter_ritz(ctx, Xd, Xd.clone(), th, 4, 5.0, 1.0, 0.0)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_chfsi_reduced_filter_converges_to_fp64_residuals(precision):
    """With the residual-form filter after the first iteration, the FP32 and mixed filters (with
    the double-float Rayleigh-Ritz apply and Gram/rotations) drive the 64 lowest residuals of
    the 32-atom cluster to the FP64 criterion 1e-8 (tighter than the 1e-5 set for reduced
    filters), and their Ritz values land within 1e-9 Ha of the all-FP64 ChFSI."""
    torch, cs = need_gpu()
    w = W.erf_cluster_32()
    ctx = make_ctx(w)
    X0 = to_dev(w.x_block())
    v0 = torch.tensor(W.gaussian(2003, ctx.d), device="cuda")
    th64 = torch.empty(w.n_s, dtype=torch.float64, device="cuda")
    r64 = torch.empty_like(th64)
    it64 = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, th64, r64, tol=1e-8,
                       max_iter=80, precision=cs.CS_FP64)
    cs.cs_set_rr_precision(ctx, cs.CS_DF64)
    cs.cs_set_dense_precision(ctx, cs.CS_DF64)
    prec = cs.CS_FP32 if precision == "fp32" else cs.CS_MIXED_BF16
    thr = torch.empty_like(th64)
    rr = torch.empty_like(th64)
    it = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, thr, rr, tol=1e-8,
                     max_iter=it64 + 10, precision=prec)
    dev = np.max(np.abs(thr.cpu().numpy()[:w.n_want] - th64.cpu().numpy()[:w.n_want]))
    print(f"{precision}: {it} iterations (FP64 {it64}), max |dtheta| {dev:.3e}, max residual "
          f"{float(rr.cpu().numpy()[:w.n_want].max()):.3e}")
    assert float(rr.cpu().numpy()[:w.n_want].max()) <= 1e-8
    assert dev < 1e-9, dev
