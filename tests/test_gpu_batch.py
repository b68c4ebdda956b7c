"""Batched filter (many clusters of uneven size in one persistent launch per Chebyshev step)
against the same clusters filtered one by one through cs_cheb_filter, and against the FP64
oracle filter; the tuner restores the blocks and keeps results unchanged."""
import numpy as np
import pytest

import workloads as W
from oracle import eigen
from tests.gpu_common import make_ctx, need_gpu, oracle_H, register, rel_errors, to_dev, to_host

pytestmark = pytest.mark.gpu


def _clusters():
    return [
        W.small_cluster(lmax=6, nmax=8, n_r=20, n_theta=14, n_phi=28, n_s=13, seed=8001),
        W.small_cluster(lmax=9, nmax=12, n_r=24, n_theta=20, n_phi=38, n_s=7, seed=8011),
        W.small_cluster(lmax=4, nmax=6, n_r=12, n_theta=10, n_phi=18, n_s=21, seed=8021),
        W.small_cluster(lmax=12, nmax=10, n_r=20, n_theta=24, n_phi=48, n_s=5, seed=8031,
                        natoms=5),
        # lmax 32: the register-blocked angular block does not fit, the row-pair block runs
        W.small_cluster(lmax=32, nmax=4, n_r=8, n_theta=64, n_phi=128, n_s=9, seed=8041,
                        natoms=3),
        # 112 radial nodes: seven rows per thread in the synthesis tiles; 130 states
        W.small_cluster(lmax=5, nmax=56, n_r=112, n_theta=12, n_phi=24, n_s=130, seed=8051,
                        R=12.0, natoms=4),
    ]


def _bounds(ctx, cs, torch):
    v0 = torch.tensor(W.gaussian(17, ctx.d), device="cuda")
    b, tmin = cs.cs_lanczos_bound(ctx, v0, 10)
    return tmin + 0.2 * (b - tmin), b, tmin


@pytest.mark.parametrize("variant,precision", [("persistent_rp4", "fp32"),
                                               ("persistent_rp2", "fp32"), ("staged", "fp32"),
                                               ("concurrent", "fp32"), ("concurrent", "mixed")])
def test_batched_filter_equals_single_cluster_filters(variant, precision):
    """One persistent launch per step (row-pair tiles of 4 or 2 states), the staged form (one
    launch per stage and tile shape) and the concurrent form (the single-cluster kernels on
    parallel graph branches, FP32 and the split-BF16 tensor-core mixed mode): all bitwise
    equal to the single-cluster filters of the same precision."""
    torch, cs = need_gpu()
    ws = _clusters()
    ctxs = [make_ctx(w) for w in ws]
    degree = 7
    prec = cs.CS_FP32 if precision == "fp32" else cs.CS_MIXED_BF16
    bounds = [_bounds(c, cs, torch) for c in ctxs]
    Xs = [to_dev(w.x_block(), dtype=torch.float32, ld=c.d + 2) for w, c in zip(ws, ctxs)]
    refs = []
    for X, c, (a, b, a0) in zip(Xs, ctxs, bounds):
        Y = X.clone()
        cs.cs_cheb_filter(c, Y, degree, a, b, a0, prec)
        refs.append(Y)
    batch = cs.cs_batch_create(ctxs, [w.n_s for w in ws], degree)
    if precision == "mixed":
        cs.cs_batch_set_precision(batch, cs.CS_MIXED_BF16)
    cs.cs_batch_set_variant(batch, variant)
    a, b, a0 = zip(*bounds)
    Yb = [X.clone() for X in Xs]
    cs.cs_batch_cheb_filter(batch, Yb, a, b, a0)
    torch.cuda.synchronize()
    for Y, R in zip(Yb, refs):
        assert torch.equal(Y, R)  # same kernels, same reduction order: bitwise equal
    assert all(cs.cs_device_error(c) == 0 for c in ctxs)
    # second call (graph replay) with new bounds gives the single-cluster results again
    a2 = [x + 0.1 for x in a]
    Yb2 = [X.clone() for X in Xs]
    cs.cs_batch_cheb_filter(batch, Yb2, a2, b, a0)
    torch.cuda.synchronize()
    for X, c, aa, bb, aa0, Y in zip(Xs, ctxs, a2, b, a0, Yb2):
        R = X.clone()
        cs.cs_cheb_filter(c, R, degree, aa, bb, aa0, prec)
        torch.cuda.synchronize()
        assert torch.equal(Y, R)
    if precision == "mixed":
        with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
            cs.cs_batch_set_variant(batch, "staged")


def test_batched_filter_vs_oracle_and_tuner():
    torch, cs = need_gpu()
    ws = _clusters()
    ctxs = [make_ctx(w) for w in ws]
    degree = 6
    bounds = [_bounds(c, cs, torch) for c in ctxs]
    a, b, a0 = zip(*bounds)
    Xs = [to_dev(w.x_block(), dtype=torch.float32) for w in ws]
    batch = cs.cs_batch_create(ctxs, [w.n_s for w in ws], degree)
    keep = [X.clone() for X in Xs]
    variant, ms = cs.cs_batch_tune(batch, Xs, a, b, a0)
    assert variant >= 0 and ms > 0
    times = cs.cs_batch_tune_times(batch)
    assert all(t > 0 for t in times.values()), times
    for X, K in zip(Xs, keep):
        assert torch.equal(X, K)  # restored
    cs.cs_batch_cheb_filter(batch, Xs, a, b, a0)
    torch.cuda.synchronize()
    for w, X, aa, bb, aa0 in zip(ws[:2], Xs[:2], a, b, a0):
        register(w)
        Hh = oracle_H(w.name)
        ref = eigen.cheb_filter(Hh.apply, w.x_block(), degree, aa, bb, aa0)
        fro, _ = rel_errors(to_host(X, Hh.basis.d), ref)
        assert fro <= 1e-4, fro
