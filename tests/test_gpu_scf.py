"""SCF pieces on the GPU (include/cs_scf.h) against the oracle (oracle/scf.py) on the same
seeded inputs: density (several chunks of states and a ragged tail), Hartree potential,
LDA, grid integrals, Anderson mixing, and the SCF loop of a small cluster."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import scf as O
from oracle.basis import Basis
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def _basis_pair(R, lmax, N, n_r, n_t, n_p):
    torch, cs = need_gpu()
    ctx = cs.cs_basis_init(R, lmax, N, n_r, n_t, n_p, 0, 0)
    return torch, cs, ctx, Basis(R, lmax, N, n_r, n_t, n_p)


def _grid(torch, a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel()),
                        device="cuda")


def _gauss(b, a, sig, Q):
    xyz = b.points()
    d = np.linalg.norm(xyz - np.asarray(a)[None, :], axis=1)
    return Q * (2 * math.pi * sig ** 2) ** -1.5 * np.exp(-d ** 2 / (2 * sig ** 2))


@pytest.mark.parametrize("n_s", [5, 37])
def test_density_matches_oracle(n_s):
    torch, cs, ctx, b = _basis_pair(8.0, 6, 8, 20, 14, 28)
    X = W.gaussian_block(9100 + n_s, b.d, n_s)
    occ = W.uniform(9200 + n_s, n_s)
    ref = O.density(b, X, occ).ravel()
    Xd = torch.zeros((n_s, b.d + 3), dtype=torch.float64, device="cuda")
    Xd[:, :b.d] = torch.tensor(X.T.copy(), device="cuda")
    rho = torch.empty(b.n_grid, dtype=torch.float64, device="cuda")
    cs.cs_density(ctx, Xd, _grid(torch, occ), rho)
    got = rho.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_hartree_matches_oracle_and_gaussian_potential():
    from scipy.special import erf
    torch, cs, ctx, b = _basis_pair(8.0, 12, 24, 48, 26, 50)
    a = np.array([0.5, -0.3, 0.4])
    rho = _gauss(b, a, 1.0, 3.0)
    vh = torch.empty(b.n_grid, dtype=torch.float64, device="cuda")
    cs.cs_hartree(ctx, _grid(torch, rho), vh)
    got = vh.cpu().numpy()
    ref = O.hartree(b, rho.reshape(b.n_r, b.n_theta, b.n_phi)).ravel()
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
    d = np.linalg.norm(b.points() - a[None, :], axis=1)
    exact = 3.0 * erf(d / math.sqrt(2.0)) / d
    assert np.max(np.abs(got - exact)) <= 1e-10 * np.max(np.abs(exact))


def test_hartree_of_random_density_matches_oracle():
    """A density with content at every l (random coefficients) on an unresolved grid."""
    torch, cs, ctx, b = _basis_pair(7.0, 6, 10, 20, 14, 28)
    rho = b.inverse_transform(W.gaussian_block(9301, b.d, 1))[..., 0].ravel()
    vh = torch.empty(b.n_grid, dtype=torch.float64, device="cuda")
    cs.cs_hartree(ctx, _grid(torch, rho), vh)
    ref = O.hartree(b, rho.reshape(b.n_r, b.n_theta, b.n_phi)).ravel()
    assert np.max(np.abs(vh.cpu().numpy() - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_lda_and_integrals_match_oracle():
    torch, cs, ctx, b = _basis_pair(8.0, 6, 8, 20, 14, 28)
    rho = 10.0 ** (-6 + 8 * W.uniform(9401, b.n_grid))  # rs from about 0.03 to 60
    rho[::97] = 0.0
    e_ref, v_ref = O.lda_xc(rho)
    exc = torch.empty(b.n_grid, dtype=torch.float64, device="cuda")
    vxc = torch.empty_like(exc)
    rd = _grid(torch, rho)
    cs.cs_lda_xc(ctx, rd, exc, vxc)
    nz = rho > 0
    for got, ref in ((exc.cpu().numpy(), e_ref), (vxc.cpu().numpy(), v_ref)):
        assert np.all(got[~nz] == 0.0)
        assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) <= 1e-13
    f2 = W.gaussian(9402, b.n_grid)
    I = cs.cs_grid_integrals(ctx, [rd, rd, _grid(torch, f2)], [exc, None, _grid(torch, f2)])
    ref = [O.integral(b, rho, e_ref), O.integral(b, rho), O.integral(b, f2, f2)]
    for x, y in zip(I, ref):
        assert abs(x - y) <= 1e-12 * abs(y)


def test_anderson_mixer_matches_oracle():
    torch, cs, ctx, b = _basis_pair(6.0, 3, 4, 10, 8, 14)
    for history in (0, 3):
        m = cs.cs_mixer_create(ctx, 0.3, history)
        ref = O.Anderson(b.weights(), 0.3, history)
        x = W.gaussian(9500, b.n_grid)
        for it in range(7):
            # a contractive map with a grid-dependent fixed point
            g = 0.5 * x + 0.3 * np.sin(x) + W.gaussian(9510 + it % 2, b.n_grid) * 0.1
            xr = ref.mix(x, g)
            xn = torch.empty(b.n_grid, dtype=torch.float64, device="cuda")
            cs.cs_mixer_mix(m, _grid(torch, x), _grid(torch, g), xn)
            got = xn.cpu().numpy()
            assert np.max(np.abs(got - xr)) <= 1e-10 * np.max(np.abs(xr)), (history, it)
            x = xr
        m.close()


def _two_atom_scf_inputs():
    b = Basis(7.0, 4, 8, 24, 12, 24)
    atoms = np.array([[0.0, 0.0, 0.7], [0.0, 0.0, -0.7]])
    vext = W.erf_cluster_potential(b.points(), atoms, Z=2.0, rc=0.8)
    rho0 = W.gaussian_atom_density(b.points(), atoms, Z=2.0, sigma=1.0)
    return b, vext, rho0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp64_lobpcg_first"])
def test_scf_matches_oracle(prec):
    """Two Z = 2 erf pseudo-atoms (4 electrons, 6 states, kT = 1e-3 Ha): the GPU SCF (ChFSI
    with one filter pass per iteration after the first solve) reaches the oracle's fixed point
    (dense eigensolves)."""
    torch, cs = need_gpu()
    b, vext, rho0 = _two_atom_scf_inputs()
    n_s = 6
    ref = O.scf(b, vext, 4.0, rho0, n_s, kT=1e-3, beta=0.3, history=8, tol=1e-11, max_iter=80)
    assert ref["converged"]
    ctx = cs.cs_basis_init(7.0, 4, 8, 24, 12, 24, 0, 0)
    p = cs.ScfParams(n_s=n_s, n_want=n_s, degree=10,
                     filter_prec=cs.CS_FP32 if prec == "fp32" else cs.CS_FP64,
                     n_electrons=4.0, kT=1e-3, beta=0.3, history=8, first_tol=1e-8,
                     first_max_iter=60 if prec != "fp64_lobpcg_first" else 200, lanczos_k=10,
                     e_ion=0.0, first_solver=1 if prec == "fp64_lobpcg_first" else 0)
    v0 = _grid(torch, W.gaussian(9601, b.d))
    S = cs.cs_scf_create(ctx, p, _grid(torch, vext), _grid(torch, rho0), v0)
    X = torch.tensor(W.gaussian_block(9602, b.d, n_s).T.copy(), device="cuda")
    theta = torch.empty(n_s, dtype=torch.float64, device="cuda")
    resid = torch.empty_like(theta)
    reps = []
    for _ in range(80):
        reps.append(cs.cs_scf_step(S, X, theta, resid))
        if len(reps) > 2 and abs(reps[-1]["dE"]) <= 1e-11:
            break
    tol_e = 1e-5 if prec == "fp32" else 1e-9
    assert abs(reps[-1]["energy"] - ref["energy"]) <= tol_e
    rho = cs.cs_scf_grid(S, 1).cpu().numpy()
    tol_r = 1e-3 if prec == "fp32" else 1e-6
    assert np.max(np.abs(rho - ref["rho"].ravel())) <= tol_r * np.max(ref["rho"])
    occ = cs.cs_scf_occupations(S)
    assert abs(occ.sum() - 2.0) <= 1e-12
    S.close()
