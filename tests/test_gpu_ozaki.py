"""GPU parity of the slice-product FP64 products (CS_FP64_SLICED: exact BF16 products of
7-bit integer slices on the tensor cores, 8 slices per value) against the oracle's slice
product (oracle/ozaki.py), bit for bit, through the C ABI (cs_dense_gram, cs_dense_rotate);
and the ChFSI loop with its Gram matrices and rotations in this arithmetic against all-FP64.

Both sides compute the exactly rounded value of the same truncated slice sum, so any
difference is an error: a wrong digit, a lost integer in an FP32 accumulator, or a
mis-rounded combination."""
import numpy as np
import pytest

import workloads as W
from oracle import ozaki
from tests.gpu_common import make_ctx, need_gpu, to_dev, to_host

pytestmark = pytest.mark.gpu

BETA, S = 7, 8


def _columns(rng, d, n):
    """Columns of mixed magnitude and sign: Gaussian columns scaled by 2^-40 .. 2^60, one with
    entries spread over 60 binades below its maximum, one all zero, one with a power-of-two
    maximum."""
    X = rng.standard_normal((d, n)) * np.ldexp(1.0, rng.integers(-40, 61, size=n))[None, :]
    if n >= 4:
        X[:, 1] = rng.standard_normal(d) * np.ldexp(1.0, rng.integers(-60, 1, size=d))
        X[:, 2] = 0.0
        X[:, 3] = rng.standard_normal(d) * 0.25
        X[d // 2, 3] = -2.0
    return X


def _ctx_for(d_min):
    """A context whose basis size d is at least d_min (the products take d from it)."""
    for lmax, nmax in ((3, 8), (6, 8), (10, 16), (20, 48), (30, 48)):
        if (lmax + 1) ** 2 * nmax >= d_min:
            w = W.small_cluster(lmax=lmax, nmax=nmax, n_r=2 * nmax, n_theta=lmax + 2,
                                n_phi=2 * lmax + 4, n_s=4)
            return make_ctx(w, with_potential=False)
    raise ValueError(d_min)


def _gram(torch, cs, ctx, A, B):
    Ad = to_dev(A, ld=ctx.d + 3)
    Bd = Ad if B is A else to_dev(B, ld=ctx.d + 1)
    C = torch.zeros((B.shape[1], A.shape[1] + 2), dtype=torch.float64, device="cuda")
    cs.cs_dense_gram(ctx, Ad, Bd, C)
    torch.cuda.synchronize()
    return C[:, :A.shape[1]].cpu().numpy().T


@pytest.mark.parametrize("shape", [(46128, 80, 80, True), (46128, 80, 80, False),
                                   (392, 13, 13, True), (1936, 37, 5, False),
                                   (1936, 130, 70, False), (392, 200, 200, True),
                                   (1936, 300, 300, True)])
def test_slice_gram_matches_oracle_bit_for_bit(shape):
    """X^T X and X^T Y of the 32-atom cluster's size (91 windows of 512 rows, K split over
    CTAs, partial sums added in 64-bit integers), one window (the single-pass path), and
    ragged shapes with several tiles on both sides. X^T X computes only the tiles that reach
    its upper triangle and mirrors them: 200 and 300 columns skip tiles, in the single-pass
    path (one window) and in the K-split path (four windows)."""
    torch, cs = need_gpu()
    d, na, nb, same = shape
    ctx = _ctx_for(d)
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    rng = np.random.default_rng(d + na + nb)
    A = np.zeros((ctx.d, na))
    A[:d] = _columns(rng, d, na)
    B = A if same else np.zeros((ctx.d, nb))
    if not same:
        B[:d] = _columns(rng, d, nb)
        B[:, 0] = A[:, min(1, na - 1)]
    got = _gram(torch, cs, ctx, A, B)
    ref = ozaki.gram(A, B, BETA, S)
    bad = np.argwhere(got.view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, (len(bad), bad[:5], got[tuple(bad[0])], ref[tuple(bad[0])])
    assert cs.cs_device_error(ctx) == 0


@pytest.mark.parametrize("shape", [(1936, 80, 80), (1936, 13, 7), (1936, 600, 40)])
def test_slice_rotation_matches_oracle_bit_for_bit(shape):
    """X Q with one exponent per row of X: the oracle's gram(X^T, Q). K = 80 (one window),
    ragged, and K = 600 (two windows in one CTA)."""
    torch, cs = need_gpu()
    d, k, n = shape
    ctx = _ctx_for(d)
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    rng = np.random.default_rng(d + k + n + 1)
    X = np.zeros((ctx.d, k))
    X[:d] = rng.standard_normal((d, k)) * np.ldexp(1.0, rng.integers(-30, 31, size=d))[:, None]
    X[d // 3] = 0.0  # an all-zero row
    Q = rng.standard_normal((k, n)) * np.ldexp(1.0, rng.integers(-8, 9, size=n))[None, :]
    Xd = to_dev(X, ld=ctx.d + 2)
    Qd = torch.tensor(np.ascontiguousarray(Q.T), device="cuda")  # (n, k): column j of Q per row
    Cd = torch.zeros((n, ctx.d + 4), dtype=torch.float64, device="cuda")
    cs.cs_dense_rotate(ctx, Xd, Qd, Cd)
    torch.cuda.synchronize()
    got = to_host(Cd, ctx.d)
    ref = ozaki.gram(X.T, Q, BETA, S)
    bad = np.argwhere(got.view(np.int64) != ref.view(np.int64))
    assert bad.size == 0, (len(bad), bad[:5])
    assert cs.cs_device_error(ctx) == 0


def test_slice_products_at_the_400_atom_size_against_fp64():
    """880 columns over d = 357216 (the 400-atom cluster's block): the Gram matrix against an
    FP64 product to its own rounding level, on sampled entries computed in exact arithmetic."""
    torch, cs = need_gpu()
    from fractions import Fraction
    w = W.erf_cluster_400_kb()
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi, 0, 0)
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(880)
    X = torch.randn((880, ctx.d), generator=gen, dtype=torch.float64, device="cuda")
    C = torch.empty((880, 880), dtype=torch.float64, device="cuda")
    cs.cs_dense_gram(ctx, X, X, C)
    torch.cuda.synchronize()
    Xh = X.cpu().numpy()
    for (i, j) in ((0, 0), (3, 877), (879, 440), (512, 511)):
        exact = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(Xh[i], Xh[j])),
                    Fraction(0))
        scale = float(np.abs(Xh[i]) @ np.abs(Xh[j]))
        assert abs(float(C[j, i]) - float(exact)) <= 8 * 2.0 ** -53 * scale, (i, j)
    assert cs.cs_device_error(ctx) == 0


def test_chfsi_with_slice_product_dense_steps():
    """The mixed filter (residual form) with the double-float Rayleigh-Ritz apply and the
    Gram matrices and rotations as slice products: on the 32-atom cluster the 64 lowest
    residuals reach 1e-8 and the Ritz values sit within 1e-9 Ha of the all-FP64 ChFSI."""
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
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    th = torch.empty_like(th64)
    rr = torch.empty_like(th64)
    it = cs.cs_chfsi(ctx, X0.clone(), w.n_want, w.degree, v0, th, rr, tol=1e-8,
                     max_iter=it64 + 10, precision=cs.CS_MIXED_BF16)
    dev = float(np.max(np.abs(th.cpu().numpy()[:w.n_want] - th64.cpu().numpy()[:w.n_want])))
    print(f"slice-product dense steps: {it} iterations (FP64 {it64}), max |dtheta| {dev:.3e}")
    assert float(rr[:w.n_want].max()) <= 1e-8
    assert dev < 1e-9, dev
    assert cs.cs_device_error(ctx) == 0
