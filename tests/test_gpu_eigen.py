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


@pytest.mark.parametrize("precision", ["fp64", "df64"])
@pytest.mark.parametrize("degree", [1, 2, 9])
def test_cheb_filter_fp64_matches_oracle(degree, precision):
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    a, b, a0, _ = _bounds(Hh)
    X = w.x_block()
    ref = eigen.cheb_filter(Hh.apply, X, degree, a, b, a0)
    Xd = to_dev(X, ld=ctx.d + 5)
    cs.cs_cheb_filter(ctx, Xd, degree, a, b, a0,
                      cs.CS_FP64 if precision == "fp64" else cs.CS_DF64)
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


@pytest.mark.parametrize("dense", ["fp64", "sliced"])
@pytest.mark.parametrize("n_s", [200, 333])
def test_cholqr_large_block_matches_oracle(n_s, dense):
    """Blocks whose Cholesky factor does not fit one CTA's shared memory take the blocked
    factor (panels of 32 columns, trailing updates over the GPU); 333 states leave a ragged
    last panel. Column norms spread over 4 decades. With slice-product dense steps the Gram
    matrix X^T X is computed on the tiles that reach its upper triangle and mirrored, and the
    rotation by the upper-triangular R^-1 stops each tile's contraction at its last column."""
    torch, cs = need_gpu()
    ctx = make_ctx(HO)
    if dense == "sliced":
        cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    rng = np.random.default_rng(81)
    X = rng.standard_normal((ctx.d, n_s)) @ np.diag(np.logspace(0, 4, n_s))
    ref = eigen.cholqr(X)
    Xd = to_dev(X)
    cs.cs_cholqr(ctx, Xd)
    torch.cuda.synchronize()
    got = to_host(Xd, ctx.d)
    assert np.max(np.abs(got.T @ got - np.eye(n_s))) < 1e-13
    assert np.max(np.abs(got - ref)) < 1e-10
    assert cs.cs_device_error(ctx) == 0


def test_cholqr_large_block_rank_deficient_reports_breakdown():
    torch, cs = need_gpu()
    ctx = make_ctx(HO)
    rng = np.random.default_rng(82)
    X = rng.standard_normal((ctx.d, 200))
    X[:, 150] = 0.0  # a zero column: its Gram diagonal is zero, the blocked factor stops
    with pytest.raises(cs.CsError, match="CS_ERR_CHOLESKY"):
        cs.cs_cholqr(ctx, to_dev(X))


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


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_chfsi_reduced_rayleigh_ritz_apply(precision):
    """Rayleigh-Ritz on an FP32 / split-BF16 H X (cs_set_rr_precision; the projection,
    eigensolve, rotations and residual norms stay FP64). The reduced H X perturbs the operator
    by about 1e-6 |H| (FP32 tables and sums; split BF16 adds its 2^-17 operand error), so the
    residuals level off and the Ritz values carry that perturbation: the solves run a fixed
    number of iterations and the Ritz values are held to the accuracy measured for each
    precision (FP32: 3.1e-6 Ha on the 32-atom cluster, |H| about 100 Ha), against the exact
    oscillator levels and the all-FP64 ChFSI. This is why the FP64 apply is the default."""
    torch, cs = need_gpu()
    prec = {"fp32": cs.CS_FP32, "mixed": cs.CS_MIXED_BF16}[precision]
    bound_ho, bound_c = {"fp32": (1e-6, 1e-5), "mixed": (1e-5, 1e-4)}[precision]
    w = HO
    ctx = make_ctx(w)
    cs.cs_set_rr_precision(ctx, prec)
    Xd = to_dev(w.x_block())
    theta = torch.empty(w.n_s, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    v0 = torch.tensor(W.gaussian(99, ctx.d), device="cuda")
    cs.cs_chfsi(ctx, Xd, w.n_want, w.degree, v0, theta, resid, tol=1e-12, max_iter=40,
                precision=prec, raise_not_converged=False)
    lev = np.loadtxt(__file__.replace("test_gpu_eigen.py", "golden/ho_levels.txt"))
    dev_ho = np.max(np.abs(theta.cpu().numpy()[:10] - lev))

    w = W.erf_cluster_32()
    ctx = make_ctx(w)
    X0 = to_dev(w.x_block())
    v0 = torch.tensor(W.gaussian(2003, ctx.d), device="cuda")
    th64 = torch.empty(w.n_s, dtype=torch.float64, device="cuda")
    r64 = torch.empty_like(th64)
    X64 = X0.clone()
    it64 = cs.cs_chfsi(ctx, X64, w.n_want, w.degree, v0, th64, r64, tol=1e-8, max_iter=80,
                       precision=cs.CS_FP64)
    cs.cs_set_rr_precision(ctx, prec)
    thr = torch.empty_like(th64)
    rr = torch.empty_like(th64)
    Xr = X0.clone()
    cs.cs_chfsi(ctx, Xr, w.n_want, w.degree, v0, thr, rr, tol=1e-12, max_iter=it64 + 10,
                precision=prec, raise_not_converged=False)
    dev = np.max(np.abs(thr.cpu().numpy()[:w.n_want] - th64.cpu().numpy()[:w.n_want]))
    floor = float(rr.cpu().numpy()[:w.n_want].max())
    print(f"{precision}: oscillator max |dtheta| {dev_ho:.3e}; 32-atom cluster: FP64 "
          f"iterations {it64}, max |dtheta| {dev:.3e}, residual floor {floor:.3e}")
    assert dev_ho < bound_ho, dev_ho
    assert floor < 1e-2, floor
    assert dev < bound_c, dev


def test_chfsi_double_float_rayleigh_ritz_holds_fp64_bars():
    """Rayleigh-Ritz H X in double-float (cs_set_rr_precision CS_DF64). All-double-float
    ChFSI (filter too) converges to residuals of 1e-8 with the oscillator's ten lowest levels
    within 1e-9 Ha of the dense oracle eigenvalues. With the FP32 filter the subspace carries
    the FP32 filter's noise only in its first iteration: after it the filter runs in residual
    form, and the FP32-filter run reaches the same 1e-8 residuals, with the Ritz values within
    1e-9 Ha: checked on the oscillator against the dense oracle and on the 32-atom cluster
    against the all-FP64 ChFSI."""
    torch, cs = need_gpu()
    w = HO
    lam = np.linalg.eigvalsh(oracle_H(w.name).dense())
    for filt, tol in ((cs.CS_DF64, 1e-8), (cs.CS_FP32, 1e-5)):
        ctx = make_ctx(w)
        cs.cs_set_rr_precision(ctx, cs.CS_DF64)
        Xd = to_dev(w.x_block())
        theta = torch.empty(w.n_s, dtype=torch.float64, device="cuda")
        resid = torch.empty_like(theta)
        v0 = torch.tensor(W.gaussian(99, ctx.d), device="cuda")
        cs.cs_chfsi(ctx, Xd, w.n_want, w.degree, v0, theta, resid, tol=tol, max_iter=80,
                    precision=filt)
        th = theta.cpu().numpy()[:10]
        assert np.max(np.abs(th - lam[:10])) < 1e-9, (filt, np.max(np.abs(th - lam[:10])))

    w = W.erf_cluster_32()
    ctx = make_ctx(w)
    X0 = to_dev(w.x_block())
    v0 = torch.tensor(W.gaussian(2003, ctx.d), device="cuda")
    th64 = torch.empty(w.n_s, dtype=torch.float64, device="cuda")
    r64 = torch.empty_like(th64)
    it64 = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, th64, r64, tol=1e-8,
                       max_iter=80, precision=cs.CS_FP64)
    cs.cs_set_rr_precision(ctx, cs.CS_DF64)
    for filt in (cs.CS_DF64, cs.CS_FP32):
        thr = torch.empty_like(th64)
        rr = torch.empty_like(th64)
        it = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, thr, rr, tol=1e-8,
                         max_iter=it64 + 10, precision=filt)
        dev = np.max(np.abs(thr.cpu().numpy()[:w.n_want] - th64.cpu().numpy()[:w.n_want]))
        floor = float(rr.cpu().numpy()[:w.n_want].max())
        print(f"filter {filt}: {it} iterations (FP64: {it64}), max |dtheta| vs FP64 "
              f"{dev:.3e}, max residual {floor:.3e}")
        assert dev < 1e-9, (filt, dev)


def test_chfsi_double_float_gram_and_rotations():
    """Cholesky-QR and Rayleigh-Ritz Gram matrices and block rotations in double-float
    (cs_set_dense_precision CS_DF64), with the double-float Rayleigh-Ritz apply: the
    all-double-float ChFSI of the 32-atom cluster and the FP32-filter one (residual form after
    the first iteration) reach residuals of 1e-8 within the FP64 solve's iterations plus ten,
    with their 64 lowest Ritz values within 1e-9 Ha of the all-FP64 ChFSI."""
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
    for filt in (cs.CS_DF64, cs.CS_FP32):
        thr = torch.empty_like(th64)
        rr = torch.empty_like(th64)
        it = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, thr, rr, tol=1e-8,
                         max_iter=it64 + 10, precision=filt)
        dev = np.max(np.abs(thr.cpu().numpy()[:w.n_want] - th64.cpu().numpy()[:w.n_want]))
        print(f"dense df64, filter {filt}: {it} iterations (FP64: {it64}), max |dtheta| "
              f"{dev:.3e}, max residual {float(rr.cpu().numpy()[:w.n_want].max()):.3e}")
        assert dev < 1e-9, (filt, dev)


def test_chfsi_mixed_filter_meets_eigenvalue_gate():
    """The mixed form (split-BF16 radial, phi and projector contractions, FP32 elsewhere in the
    filter; residual form after the first iteration) with the double-float Rayleigh-Ritz apply
    and Gram/rotations: on the 32-atom cluster the run meets the reduced-precision criterion
    (residuals <= 1e-5) within the FP64 solve's iterations plus ten, and the 64 lowest Ritz
    values land within 1e-6 Ha of the all-FP64 ChFSI (the acceptance gate of the
    mixed-precision form)."""
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
    thr = torch.empty_like(th64)
    rr = torch.empty_like(th64)
    it = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, thr, rr, tol=1e-5,
                     max_iter=it64 + 10, precision=cs.CS_MIXED_BF16)
    dev = np.max(np.abs(thr.cpu().numpy()[:w.n_want] - th64.cpu().numpy()[:w.n_want]))
    print(f"mixed filter: {it} iterations to 1e-5, max |dtheta| vs FP64 {dev:.3e}")
    assert float(rr.cpu().numpy()[:w.n_want].max()) <= 1e-5
    assert dev < 1e-6, dev


@pytest.mark.parametrize("dense", ["fp64", "sliced"])
def test_rayleigh_ritz_large_block_matches_oracle(dense):
    """A 300-state block (the projected matrix's tridiagonal solve no longer fits one CTA's
    shared memory, so the device-wide FP32 stage runs before the FP64 refinement): Ritz values
    and residual norms against the oracle's Rayleigh-Ritz, on the oscillator basis (d = 1936).
    With slice-product dense steps the Gram matrix, the rotations and the refinement's 300 x 300
    products (above 256 states) are slice products on the tensor cores."""
    torch, cs = need_gpu()
    w = HO
    ctx = make_ctx(w)
    if dense == "sliced":
        cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    Hh = oracle_H(w.name)
    X = eigen.cholqr(W.gaussian_block(4300, ctx.d, 300))
    th_ref, X_ref, _, res_ref = eigen.rayleigh_ritz(Hh.apply, X)
    Xd = to_dev(X)
    theta = torch.empty(300, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    cs.cs_rayleigh_ritz(ctx, Xd, theta, resid)
    torch.cuda.synchronize()
    th = theta.cpu().numpy()
    print(f"n_s 300: max |dtheta| {np.max(np.abs(th - th_ref)):.3e}, |theta| max "
          f"{np.abs(th_ref).max():.3e}")
    assert np.max(np.abs(th - th_ref)) < 1e-11 * np.abs(th_ref).max()
    assert np.max(np.abs(resid.cpu().numpy() - res_ref)) < 1e-10 * np.abs(res_ref).max()
    got = to_host(Xd, ctx.d)
    assert np.max(np.abs(got.T @ got - np.eye(300))) < 1e-12
    assert cs.cs_device_error(ctx) == 0
