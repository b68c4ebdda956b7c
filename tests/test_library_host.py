"""The C-ABI library without a GPU: it loads, exports every entry point that include/*.h
declare, builds its host tables (compared here with the oracle's, which share no code
with them), and rejects bad arguments and device calls on a host-only context."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    cs = pytest.importorskip("paper_1404_3773_gb300")
    return cs


def _declared_symbols():
    import glob
    names = set()
    for path in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        hdr = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"\b(cs_[a-z_0-9]+)\s*\(", hdr))
    return sorted(names)


def test_header_symbols_exported():
    cs = _lib()
    lib = ctypes.CDLL(cs.library_path())
    names = _declared_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    # the binding mirrors every declared entry point under the same name
    for n in names:
        assert hasattr(cs, n), n


@pytest.mark.parametrize("rule", [0, 1])
def test_host_tables_match_oracle(rule):
    cs = _lib()
    from oracle.basis import Basis
    ctx = cs.cs_basis_init(14.0, 30, 48, 96, 60, 120, rule, -1)
    b = Basis(14.0, 30, 48, 96, 60, 120, ["gauss_legendre", "gauss_jacobi_r2"][rule])
    r, wr, t, wt, ph = cs.cs_grid(ctx)
    assert np.max(np.abs(r - b.r)) < 1e-13
    assert np.max(np.abs(wr - b.w_r) / b.w_r) < 1e-12
    assert np.max(np.abs(t - b.t)) < 1e-15 and np.max(np.abs(wt - b.w_t)) < 1e-14
    assert np.max(np.abs(ph - b.phi)) < 1e-15
    z = cs.cs_bessel_zeros(ctx, 30, 48)
    assert np.max(np.abs(z - b.z) / b.z) < 1e-14
    hl = cs.cs_kinetic(ctx)
    assert np.max(np.abs(hl - b.half_lambda) / b.half_lambda) < 1e-13
    assert ctx.d == b.d == 46128


def test_bad_arguments_rejected():
    cs = _lib()
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_basis_init(8.0, 10, 16, 32, 22, 41, 0, -1)  # odd n_phi
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_basis_init(8.0, 10, 16, 32, 10, 42, 0, -1)  # n_theta <= lmax
    with pytest.raises(cs.CsError, match="CS_ERR_ARG"):
        cs.cs_basis_init(-1.0, 10, 16, 32, 22, 42, 0, -1)


def test_device_calls_on_host_context_report_state_error():
    cs = _lib()
    ctx = cs.cs_basis_init(8.0, 4, 6, 12, 10, 20, 0, -1)
    lib = ctypes.CDLL(cs.library_path())
    lib.cs_set_potential.argtypes = [ctypes.c_void_p] * 3
    assert lib.cs_set_potential(ctx.handle, None, None) == 4  # CS_ERR_STATE
    assert "no device" in cs.cs_last_error(ctx)
    lib.cs_apply_H.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.cs_apply_H(ctx.handle, 4, None, None, ctx.d, 0, None, None) == 4


def test_workspace_bytes_grows_with_block():
    cs = _lib()
    ctx = cs.cs_basis_init(8.0, 10, 16, 32, 22, 42, 0, -1)
    a = cs.cs_workspace_bytes(ctx, 8)
    b = cs.cs_workspace_bytes(ctx, 16)
    c = cs.cs_workspace_bytes(ctx, 16, cs.CS_FP32)
    assert 0 < a < b < c
    # it covers at least the radial-node intermediate, two blocks and the Lanczos basis
    assert b >= 32 * 121 * 16 * 8 + 4 * ctx.d * 16 * 8


def test_fermi_occupations_match_oracle():
    """cs_fermi_occupations (host Brent root of the electron count) against the oracle's
    (scipy brentq), including a degenerate level at the Fermi energy."""
    cs = _lib()
    from oracle import scf
    for lam, ne, kT in (([-1.0, -0.5, -0.5, 0.2, 0.9], 4.0, 1e-3),
                        (np.linspace(-2.0, 1.0, 40), 31.0, 0.05),
                        ([-0.3, -0.2], 1.0, 1e-6)):
        occ, mu, S = cs.cs_fermi_occupations(lam, ne, kT)
        f, m, S2 = scf.fermi_occupations(np.asarray(lam), ne, kT)
        assert np.max(np.abs(occ - f)) <= 1e-10
        assert abs(mu - m) <= 1e-9 and abs(S - S2) <= 1e-8
        # one ulp of mu moves the count by about ulp(mu) / (4 kT)
        assert abs(occ.sum() - ne / 2) <= 1e-12 + 1e-16 / kT


def test_atom_descriptors_match_oracle():
    cs = _lib()
    import workloads as W
    from oracle import learned_density as LD
    atoms = W.place_atoms(8850, 9, 5.0, 2.0)
    mu = np.linspace(2.0, 10.0, 16)
    got = cs.cs_atom_descriptors(atoms, mu, 0.5)
    ref = LD.descriptors(atoms, mu, 0.5)
    assert np.max(np.abs(got - ref)) <= 1e-13


def test_df64_split_of_a_double_matches_fp64_rounding(tmp_path):
    """The double-float split of a double takes an integer/FP32 path where its parts are normal
    floats and FP64 arithmetic elsewhere; both give hi = fl(x), lo = fl(x - hi) bit for bit.
    Checked by a host program built with nvcc (no GPU needed)."""
    import shutil
    import subprocess

    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = os.path.join(os.path.dirname(__file__), "native", "df64_split_check.cu")
    exe = str(tmp_path / "df64_split_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-o", exe, src], check=True,
                   capture_output=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-2000:]
