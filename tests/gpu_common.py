"""Shared set-up for the GPU tests: a library context and the oracle for one workload,
both fed from the same seeded inputs (workloads), each on its own quadrature grid."""
import functools

import numpy as np
import pytest

import workloads as W

RULES = {"gauss_legendre": 0, "gauss_jacobi_r2": 1}


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1404_3773_gb300 as cs  # raises if the library is missing
    return torch, cs


def make_ctx(w, with_potential=True, device=0):
    torch, cs = need_gpu()
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi,
                           RULES[w.radial_rule], device)
    if with_potential:
        v = w.potential_at(cs.grid_points(ctx))
        cs.cs_set_potential(ctx, torch.tensor(v, dtype=torch.float64, device=f"cuda:{device}"))
    return ctx


@functools.lru_cache(maxsize=16)
def oracle_H(w_key):
    from oracle.basis import basis_for
    from oracle.hamiltonian import Hamiltonian
    w = _WORKLOADS[w_key]
    b = basis_for(w)
    return Hamiltonian(b, w.potential_at(b.points()))


_WORKLOADS = {}


def register(w):
    old = _WORKLOADS.get(w.name)
    assert old is None or old == w, f"two different workloads named {w.name}"
    _WORKLOADS[w.name] = w
    return w.name


def to_dev(X, dtype=None, ld=None):
    """numpy (d, S) -> torch (S, ld) on cuda (row s = state s)."""
    import torch
    d, S = X.shape
    ld = d if ld is None else ld
    out = torch.zeros((S, ld), dtype=dtype or torch.float64, device="cuda")
    out[:, :d] = torch.tensor(np.ascontiguousarray(X.T), dtype=out.dtype, device="cuda")
    return out


def to_host(T, d):
    return T[:, :d].double().cpu().numpy().T.copy()


def rel_errors(got, ref):
    fro = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    col = np.max(np.max(np.abs(got - ref), axis=0) / np.linalg.norm(ref, axis=0))
    return fro, col
