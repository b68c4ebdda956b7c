"""cs_apply_H_noalloc: H.X without a caller workspace, for callers that cannot allocate
device memory when they call (their free memory is held by another allocator, or they
cannot afford cudaMalloc's device-wide synchronisation). Its scratch is an array built
into the library, so the test checks, through the C ABI, that two calls in a row agree
with cs_apply_H (the workspace entry point: bitwise, since the same kernels run) and with
the FP64 oracle within the parity tolerance, that the second call does not see the first
call's leftovers, that the caller's current device is kept, and that oversize requests
and the unsupported precisions are refused.
This file sorts last so that a run stopping at the first failure has run the rest."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import (make_ctx, need_gpu, oracle_H, register, rel_errors, to_dev,
                              to_host)

pytestmark = pytest.mark.gpu

SMALL = W.small_cluster(lmax=6, nmax=8, n_r=20, n_theta=14, n_phi=28, n_s=13)
register(SMALL)

TOL64 = 1e-11
TOL32 = 2e-5


def _reference(cs, torch, ctx, Xd, prec):
    out = torch.empty_like(Xd)
    cs.cs_apply_H(ctx, Xd, out, prec)
    torch.cuda.synchronize()
    return to_host(out, ctx.d)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_workspace_entry_point_twice(precision):
    torch, cs = need_gpu()
    w = SMALL
    ctx = make_ctx(w)
    Hh = oracle_H(w.name)
    prec = cs.CS_FP64 if precision == "fp64" else cs.CS_FP32
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = TOL64 if precision == "fp64" else TOL32
    dev_before = torch.cuda.current_device()
    # first call: 13 states
    Xa_h = w.x_block(13)
    Xa = to_dev(Xa_h, dtype=dt, ld=ctx.d + 3)
    HXa = torch.zeros_like(Xa)
    cs.cs_apply_H_noalloc(ctx, Xa, HXa, prec)
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == dev_before
    got = to_host(HXa, ctx.d)
    # the workspace entry point runs the same kernels on the same block: bitwise equal
    assert np.array_equal(got, _reference(cs, torch, ctx, Xa, prec))
    # and the FP64 oracle on the block as the GPU saw it
    fro, col = rel_errors(got, Hh.apply(to_host(Xa, ctx.d)))
    assert fro <= tol and col <= tol, (fro, col)
    # second call right after, different states and a different block size: the
    # scratch keeps the first call's contents, which must not leak into this result
    Xb = to_dev(W.gaussian_block(777, ctx.d, 5), dtype=dt)
    HXb = torch.zeros_like(Xb)
    cs.cs_apply_H_noalloc(ctx, Xb, HXb, prec)
    torch.cuda.synchronize()
    got = to_host(HXb, ctx.d)
    assert np.array_equal(got, _reference(cs, torch, ctx, Xb, prec))
    fro, col = rel_errors(got, Hh.apply(to_host(Xb, ctx.d)))
    assert fro <= tol and col <= tol, (fro, col)


@pytest.mark.parametrize("precision", ["mixed", "df64"])
def test_noalloc_refuses_staged_precisions(precision):
    torch, cs = need_gpu()
    ctx = make_ctx(SMALL)
    prec = cs.CS_MIXED_BF16 if precision == "mixed" else cs.CS_DF64
    dt = torch.float32 if precision == "mixed" else torch.float64
    X = to_dev(SMALL.x_block(3), dtype=dt)
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_apply_H_noalloc(ctx, X, torch.empty_like(X), prec)
    assert "CS_FP64 or CS_FP32" in cs.cs_last_error(ctx)


def test_noalloc_rejects_blocks_larger_than_its_scratch():
    torch, cs = need_gpu()
    ctx = make_ctx(SMALL)
    # 20 radial nodes x 49 (l,m) x 8 bytes = 7840 bytes per state: 5000 states > 32 MiB
    X = torch.zeros((5000, ctx.d), dtype=torch.float64, device="cuda")
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_apply_H_noalloc(ctx, X, torch.empty_like(X), cs.CS_FP64)
    assert "exceeds the static scratch" in cs.cs_last_error(ctx)
