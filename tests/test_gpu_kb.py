"""Kleinman-Bylander projector pair (Sec. 2.3.2) in every precision against the FP64 oracle,
through the C ABI, and the 400-atom lmax-60 cluster with projectors at full size.

The library forward-transforms the projector functions sampled on its own grid
(cs_forward_transform) and takes the coefficients through cs_set_projectors; the oracle
forward-transforms the same functions on its own grid. Bars: FP64 1e-11 (Frobenius and
per column, relative); FP32 2e-5; mixed split-BF16 1e-4 (Frobenius)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_common import RULES, make_ctx, need_gpu, oracle_H, register, rel_errors, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-11, 1e-11), "fp32": (2e-5, 2e-4), "mixed": (1e-4, 1e-3)}

CASES = {
    # 2 atoms (8 projectors), 13 states: ragged K chunks of d = 392, split K over 7 CTAs
    "small_2atoms": (W.small_cluster(lmax=6, nmax=8, n_r=20, n_theta=14, n_phi=28, n_s=13,
                                     seed=7401), 2),
    # 40 atoms (160 projectors: two projector tiles, three ragged K chunks), 150 states
    # (two state tiles), d = 1936
    "ho_40atoms_150states": (W.Workload("ho_kb_l10_n16", R=8.0, lmax=10, nmax=16, n_r=32,
                                        n_theta=22, n_phi=42, radial_rule="gauss_legendre",
                                        n_s=150, degree=8, potential="ho", x_seed=7502,
                                        extra={"omega": 1.0, "center": (0.3, -0.2, 0.1)}), 40),
}
for _w, _ in CASES.values():
    register(_w)


def _prec(cs, p):
    return {"fp64": cs.CS_FP64, "fp32": cs.CS_FP32, "mixed": cs.CS_MIXED_BF16}[p]


def _set_library_projectors(torch, cs, ctx, atoms, batch=64):
    """Projector coefficients by the library's own forward transform, `batch` at a time."""
    from workloads.device import kb_couplings, kb_projector_values_t
    xyz = torch.tensor(cs.grid_points(ctx), device="cuda")
    na = atoms.shape[0]
    pcoef = torch.empty((4 * na, ctx.d), dtype=torch.float64, device="cuda")
    per = max(1, batch // 4)
    for a0 in range(0, na, per):
        cnt = min(per, na - a0)
        pg = kb_projector_values_t(xyz, atoms, rc=1.0, first=a0, count=cnt)
        pg = pg.reshape(4 * cnt, ctx.n_r, ctx.n_theta, ctx.n_phi).contiguous()
        cs.cs_forward_transform(ctx, pg, pcoef[4 * a0:4 * (a0 + cnt)])
        del pg
    cs.cs_set_projectors(ctx, pcoef, kb_couplings(na))
    torch.cuda.synchronize()


def _oracle_with_projectors(w, atoms):
    from oracle.hamiltonian import Hamiltonian
    b = oracle_H(w.name).basis
    pg_o, h = W.kb_projector_values(b.points(), atoms, rc=1.0)
    return Hamiltonian(b, oracle_H(w.name).v, pg_o, h)


def _apply(torch, cs, ctx, X, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    Xd = to_dev(X, dtype=dt, ld=ctx.d + 8)
    HXd = torch.zeros_like(Xd)
    cs.cs_apply_H(ctx, Xd, HXd, _prec(cs, prec))
    torch.cuda.synchronize()
    assert torch.all(HXd[:, ctx.d:] == 0)
    return to_host(HXd, ctx.d)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_projector_pair_matches_oracle_all_precisions(case, prec):
    torch, cs = need_gpu()
    w, natoms = CASES[case]
    atoms = W.place_atoms(w.x_seed + 11, natoms, 0.6 * w.R, 1.0)
    ctx = make_ctx(w)
    Hkb = _oracle_with_projectors(w, atoms)
    X = w.x_block()
    ref = Hkb.apply(X)
    kb_ref = ref - oracle_H(w.name).apply(X)
    _set_library_projectors(torch, cs, ctx, atoms)
    got = _apply(torch, cs, ctx, X, prec)
    fro, col = rel_errors(got, ref)
    tf, tc = TOL[prec]
    print(f"kb {case} {prec}: fro {fro:.3e} col {col:.3e}")
    assert fro <= tf and col <= tc, (fro, col)
    # the projector term alone (difference of two applies), relative to its own size; the
    # bound allows for the rounding of the epilogue sum, whose terms are about 10^3 times
    # larger than the projector term for these random blocks
    cs.cs_set_projectors(ctx, None, None)
    kb_got = got - _apply(torch, cs, ctx, X, prec)
    kfro = np.linalg.norm(kb_got - kb_ref) / np.linalg.norm(kb_ref)
    print(f"kb {case} {prec}: projector term alone {kfro:.3e}")
    assert kfro <= {"fp64": 1e-10, "fp32": 1e-3, "mixed": 1e-3}[prec], kfro
    assert cs.cs_device_error(ctx) == 0


def test_set_projectors_replaces_and_removes():
    torch, cs = need_gpu()
    w, _ = CASES["small_2atoms"]
    ctx = make_ctx(w)
    X = w.x_block()
    plain = _apply(torch, cs, ctx, X, "fp64")
    atoms = W.place_atoms(7701, 3, 3.0, 1.0)
    _set_library_projectors(torch, cs, ctx, atoms)
    _set_library_projectors(torch, cs, ctx, atoms[:1])  # replaced by a single atom
    ref = _oracle_with_projectors(w, atoms[:1]).apply(X)
    fro, _ = rel_errors(_apply(torch, cs, ctx, X, "fp64"), ref)
    assert fro <= 1e-11
    cs.cs_set_projectors(ctx, None, None)
    assert np.array_equal(_apply(torch, cs, ctx, X, "fp64"), plain)


@pytest.mark.slow
def test_erf400kb_full_size():
    """The 400-atom cluster (R = 26, lmax 60, 96 radial functions, d = 357216, 192 x 120 x
    240 grid) at full size: FP64 H.X against the oracle on two sampled state columns, without
    and with the projectors of two atoms; then all 1600 projectors on one 128-state chunk:
    mixed and FP32 against the GPU FP64 result pinned above."""
    torch, cs = need_gpu()
    from oracle.basis import basis_for
    from oracle.hamiltonian import Hamiltonian
    from workloads.device import erf_cluster_potential_t
    w = W.erf_cluster_400_kb()
    atoms = w.atoms()
    ctx = cs.cs_basis_init(w.R, w.lmax, w.nmax, w.n_r, w.n_theta, w.n_phi,
                           RULES[w.radial_rule], 0)
    assert ctx.d == 357216
    v_lib = erf_cluster_potential_t(torch.tensor(cs.grid_points(ctx), device="cuda"), atoms)
    cs.cs_set_potential(ctx, v_lib.contiguous())
    b = basis_for(w)
    v_or = erf_cluster_potential_t(torch.tensor(b.points(), device="cuda"), atoms).cpu().numpy()
    Hloc = Hamiltonian(b, v_or)
    X2 = w.x_block(2)
    ref_loc = Hloc.apply(X2)
    fro, col = rel_errors(_apply(torch, cs, ctx, X2, "fp64"), ref_loc)
    assert fro <= 1e-11 and col <= 1e-11, (fro, col)
    # projectors of two atoms, against the oracle's own forward transforms
    sub = atoms[[0, atoms.shape[0] - 1]]
    pg_o, h = W.kb_projector_values(b.points(), sub, rc=1.0)
    ref_kb = Hamiltonian(b, v_or, pg_o, h).apply(X2)
    _set_library_projectors(torch, cs, ctx, sub)
    for prec in ("fp64", "fp32", "mixed"):
        fro, col = rel_errors(_apply(torch, cs, ctx, X2, prec), ref_kb)
        print(f"erf400kb two atoms {prec}: fro {fro:.3e} col {col:.3e}")
        assert fro <= TOL[prec][0] and col <= TOL[prec][1], (prec, fro, col)
    # every projector (1600), one chunk of 128 states
    _set_library_projectors(torch, cs, ctx, atoms)
    Xc = w.x_block(128)
    y64 = _apply(torch, cs, ctx, Xc, "fp64")
    for prec in ("fp32", "mixed"):
        fro, col = rel_errors(_apply(torch, cs, ctx, Xc, prec), y64)
        print(f"erf400kb 1600 projectors, 128 states {prec}: fro {fro:.3e} col {col:.3e}")
        assert fro <= TOL[prec][0] and col <= TOL[prec][1], (prec, fro, col)
    assert cs.cs_device_error(ctx) == 0


@pytest.mark.parametrize("case", list(CASES))
def test_projector_pair_as_slice_products_matches_oracle(case):
    """With CS_FP64_SLICED dense products the FP64 H.X takes its projector pair as exact
    slice products on the tensor cores: the FP64 bar against the oracle still holds."""
    torch, cs = need_gpu()
    w, natoms = CASES[case]
    atoms = W.place_atoms(w.x_seed + 11, natoms, 0.6 * w.R, 1.0)
    ctx = make_ctx(w)
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    Hkb = _oracle_with_projectors(w, atoms)
    X = w.x_block()
    ref = Hkb.apply(X)
    _set_library_projectors(torch, cs, ctx, atoms)
    got = _apply(torch, cs, ctx, X, "fp64")
    fro, col = rel_errors(got, ref)
    print(f"kb {case} fp64 sliced: fro {fro:.3e} col {col:.3e}")
    assert fro <= 1e-11 and col <= 1e-11, (fro, col)
    assert cs.cs_device_error(ctx) == 0


@pytest.mark.parametrize("case", list(CASES))
def test_double_float_apply_with_slice_product_projectors(case):
    """CS_DF64 H.X with projectors (allowed with CS_FP64_SLICED dense products: the projector
    term is formed as exact slice products and added in double-float) against the oracle at
    the FP64 bar; without slice products the call is refused."""
    torch, cs = need_gpu()
    w, natoms = CASES[case]
    atoms = W.place_atoms(w.x_seed + 11, natoms, 0.6 * w.R, 1.0)
    ctx = make_ctx(w)
    Hkb = _oracle_with_projectors(w, atoms)
    X = w.x_block()
    ref = Hkb.apply(X)
    _set_library_projectors(torch, cs, ctx, atoms)
    Xd = to_dev(X, ld=ctx.d + 8)
    with pytest.raises(cs.CsError, match="CS_ERR_STATE"):
        cs.cs_apply_H(ctx, Xd, torch.zeros_like(Xd), cs.CS_DF64)
    cs.cs_set_dense_precision(ctx, cs.CS_FP64_SLICED)
    HXd = torch.zeros_like(Xd)
    cs.cs_apply_H(ctx, Xd, HXd, cs.CS_DF64)
    torch.cuda.synchronize()
    fro, col = rel_errors(to_host(HXd, ctx.d), ref)
    print(f"kb {case} df64 with sliced projectors: fro {fro:.3e} col {col:.3e}")
    assert fro <= 1e-11 and col <= 1e-11, (fro, col)
    assert cs.cs_device_error(ctx) == 0
