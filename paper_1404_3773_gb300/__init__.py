"""Python binding of libclusterspec: the ChFSI hot path of the spherical spectral
Kohn-Sham method on a GB300 (sm_103a).

Argument marshalling only: every numerical step runs in the library's CUDA kernels
(include/cs.h documents each entry point). PyTorch supplies device memory and streams.
There is no CPU fallback: importing this package raises if the compiled library is
missing, and every call raises RuntimeError on a non-zero cs_status.

Blocks of states are torch tensors of shape (n_s, ld) (row i = state i), i.e. the
column-major d x n_s matrices of the C ABI with leading dimension ld = tensor.stride(0);
only the first d entries of each row are used.
"""
from __future__ import annotations

import ctypes
import os

import torch  # loads the CUDA runtime that the library links against

__all__ = [
    "CS_FP64", "CS_FP32", "CS_MIXED_BF16", "CS_DF64", "CS_FP64_SLICED", "CS_RADIAL_GAUSS_LEGENDRE", "CS_RADIAL_GAUSS_JACOBI_R2",
    "CsError", "Context", "cs_basis_init", "cs_basis_free", "cs_basis_dims", "cs_grid",
    "cs_kinetic", "cs_bessel_zeros", "cs_set_potential", "cs_set_projectors",
    "cs_forward_transform", "cs_inverse_transform", "cs_workspace_bytes", "cs_apply_H",
    "cs_cheb_filter", "cs_cholqr", "cs_rayleigh_ritz", "cs_lanczos_bound", "cs_chfsi",
    "cs_chfsi_step", "cs_cheb_filter_ritz", "cs_chfsi_step_ritz", "cs_profile_begin", "cs_profile_end", "cs_apply_H_noalloc",
    "cs_set_rr_precision", "cs_set_dense_precision", "cs_dense_gram", "cs_dense_rotate",
    "cs_device_error", "Batch", "cs_batch_create", "cs_batch_free", "cs_batch_workspace_bytes",
    "cs_batch_cheb_filter", "cs_batch_tune", "cs_batch_tune_times", "cs_batch_set_variant",
    "cs_batch_set_precision",
    "cs_batch_last_error",
    "cs_last_error", "cs_launch_count", "library_path", "exported_symbols", "grid_points",
    "cs_measure_peaks",
    "cs_lobpcg_workspace_bytes", "cs_lobpcg",
    # SCF pieces (include/cs_scf.h)
    "CS_DENSITY_CHUNK", "CS_MIXER_MAX_HISTORY", "CS_GRID_INTEGRALS_MAX", "ScfParams",
    "ScfReport", "Mixer", "Scf", "cs_scf_workspace_bytes", "cs_density", "cs_hartree",
    "cs_lda_xc", "cs_grid_integrals", "cs_fermi_occupations", "cs_mixer_create",
    "cs_mixer_mix", "cs_mixer_reset", "cs_mixer_free", "cs_scf_create", "cs_scf_work_bytes",
    "cs_scf_step", "cs_scf_grid", "cs_scf_occupations", "cs_scf_free",
    # learned initial density (include/cs_learned.h)
    "Mlp", "cs_atom_descriptors", "cs_atom_density", "cs_fit_workspace_bytes",
    "cs_fit_atom_density", "cs_mlp_create", "cs_mlp_free", "cs_mlp_param_count", "cs_mlp_params",
    "cs_mlp_forward", "cs_mlp_loss_grad", "cs_mlp_train_step", "cs_mlp_last_error",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libclusterspec.so")

CS_FP64, CS_FP32, CS_MIXED_BF16, CS_DF64, CS_FP64_SLICED = 0, 1, 2, 3, 4
CS_RADIAL_GAUSS_LEGENDRE, CS_RADIAL_GAUSS_JACOBI_R2 = 0, 1
_STATUS = {0: "CS_OK", 1: "CS_ERR_ARG", 2: "CS_ERR_ALLOC", 3: "CS_ERR_CUDA",
           4: "CS_ERR_STATE", 5: "CS_ERR_CHOLESKY", 6: "CS_ERR_NOT_CONVERGED",
           7: "CS_ERR_TIMEOUT", 8: "CS_ERR_NUMERIC"}

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        f"libclusterspec.so not found at {_LIB_PATH}; build it with "
        "`python -m paper_1404_3773_gb300.build` (there is no CPU fallback)")

_lib = ctypes.CDLL(_LIB_PATH)


class _Quad(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("radial", ctypes.c_int)]


class ScfParams(ctypes.Structure):
    """cs_scf_params (include/cs_scf.h)."""
    _fields_ = [("n_s", ctypes.c_int), ("n_want", ctypes.c_int), ("degree", ctypes.c_int),
                ("filter_prec", ctypes.c_int), ("n_electrons", ctypes.c_double),
                ("kT", ctypes.c_double), ("beta", ctypes.c_double), ("history", ctypes.c_int),
                ("first_tol", ctypes.c_double), ("first_max_iter", ctypes.c_int),
                ("lanczos_k", ctypes.c_int), ("e_ion", ctypes.c_double),
                ("first_solver", ctypes.c_int)]


class ScfReport(ctypes.Structure):
    """cs_scf_report (include/cs_scf.h)."""
    _fields_ = [("iteration", ctypes.c_int), ("chfsi_iterations", ctypes.c_int),
                ("energy", ctypes.c_double), ("dE", ctypes.c_double), ("mu", ctypes.c_double),
                ("entropy", ctypes.c_double), ("band", ctypes.c_double),
                ("e_hartree", ctypes.c_double), ("e_xc", ctypes.c_double),
                ("max_resid", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_vp = ctypes.c_void_p
_i = ctypes.c_int
_ll = ctypes.c_longlong
_d = ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "cs_basis_init": (_i, [_d, _i, _i, ctypes.POINTER(_Quad), _i, ctypes.POINTER(_vp)]),
    "cs_basis_free": (_i, [_vp]),
    "cs_basis_dims": (_i, [_vp, ctypes.POINTER(_ll), ctypes.POINTER(_i), ctypes.POINTER(_i),
                           ctypes.POINTER(_i)]),
    "cs_grid": (_i, [_vp, _dp, _dp, _dp, _dp, _dp]),
    "cs_kinetic": (_i, [_vp, _dp]),
    "cs_bessel_zeros": (_i, [_vp, _dp]),
    "cs_set_potential": (_i, [_vp, _vp, _vp]),
    "cs_set_projectors": (_i, [_vp, _i, _vp, _dp, _vp]),
    "cs_forward_transform": (_i, [_vp, _i, _vp, _vp, _ll, _vp, _vp]),
    "cs_inverse_transform": (_i, [_vp, _i, _vp, _ll, _vp, _vp, _vp]),
    "cs_workspace_bytes": (_i, [_vp, _i, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_apply_H": (_i, [_vp, _i, _vp, _vp, _ll, _i, _vp, _vp]),
    "cs_cheb_filter": (_i, [_vp, _i, _vp, _ll, _i, _d, _d, _d, _i, _vp, _vp]),
    "cs_cholqr": (_i, [_vp, _i, _vp, _ll, _vp, _vp]),
    "cs_rayleigh_ritz": (_i, [_vp, _i, _vp, _ll, _vp, _vp, _vp, _vp, _vp]),
    "cs_lanczos_bound": (_i, [_vp, _i, _vp, _dp, _dp, _vp, _vp]),
    "cs_chfsi": (_i, [_vp, _i, _i, _vp, _ll, _i, _d, _i, _i, _vp, _vp, _vp,
                      ctypes.POINTER(_i), _vp, _vp]),
    "cs_apply_H_noalloc": (_i, [_vp, _i, _vp, _vp, _ll, _i, _vp]),
    "cs_chfsi_step": (_i, [_vp, _i, _vp, _ll, _i, _d, _d, _d, _i, _vp, _vp, _vp, _vp]),
    "cs_cheb_filter_ritz": (_i, [_vp, _i, _vp, _ll, _vp, _ll, _vp, _i, _d, _d, _d, _i, _vp, _vp]),
    "cs_chfsi_step_ritz": (_i, [_vp, _i, _vp, _vp, _ll, _i, _d, _d, _d, _i, _vp, _vp, _vp,
                                _vp]),
    "cs_profile_begin": (_i, [_vp]),
    "cs_device_error": (_i, [_vp, ctypes.POINTER(_i)]),
    "cs_profile_end": (_i, [_vp, _dp, ctypes.POINTER(_ll)]),
    "cs_set_rr_precision": (_i, [_vp, _i]),
    "cs_set_dense_precision": (_i, [_vp, _i]),
    "cs_dense_gram": (_i, [_vp, _i, _i, _vp, _ll, _vp, _ll, _vp, _ll, _vp, _vp]),
    "cs_dense_rotate": (_i, [_vp, _i, _i, _vp, _ll, _vp, _ll, _vp, _ll, _vp, _vp]),
    "cs_batch_create": (_i, [_i, ctypes.POINTER(_vp), ctypes.POINTER(_i), _i, ctypes.POINTER(_vp)]),
    "cs_batch_free": (_i, [_vp]),
    "cs_batch_workspace_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_batch_cheb_filter": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_ll), _dp, _dp, _dp,
                                  _vp, _vp]),
    "cs_batch_tune_times": (_i, [_vp, ctypes.POINTER(ctypes.c_float), _i]),
    "cs_batch_set_variant": (_i, [_vp, _i]),
    "cs_batch_set_precision": (_i, [_vp, _i]),
    "cs_batch_tune": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_ll), _dp, _dp, _dp, _vp, _vp,
                           ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_float)]),
    "cs_batch_last_error": (ctypes.c_char_p, [_vp]),
    "cs_last_error": (ctypes.c_char_p, [_vp]),
    "cs_measure_peaks": (_i, [_i, _dp, _dp]),
    "cs_launch_count": (_ll, [_vp]),
    "cs_lobpcg_workspace_bytes": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_lobpcg": (_i, [_vp, _i, _i, _vp, _ll, _d, _i, _i, _vp, _vp, ctypes.POINTER(_i),
                       ctypes.POINTER(_i), _vp, _vp]),
    # SCF pieces
    "cs_scf_workspace_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_density": (_i, [_vp, _i, _vp, _ll, _vp, _vp, _vp, _vp]),
    "cs_hartree": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "cs_lda_xc": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "cs_grid_integrals": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _dp, _vp, _vp]),
    "cs_fermi_occupations": (_i, [_i, _dp, _d, _d, _dp, _dp, _dp]),
    "cs_mixer_create": (_i, [_vp, _d, _i, ctypes.POINTER(_vp)]),
    "cs_mixer_mix": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "cs_mixer_reset": (_i, [_vp]),
    "cs_mixer_free": (_i, [_vp]),
    "cs_scf_create": (_i, [_vp, ctypes.POINTER(ScfParams), _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "cs_scf_work_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_scf_step": (_i, [_vp, _vp, _ll, _vp, _vp, _vp, _vp, ctypes.POINTER(ScfReport)]),
    "cs_scf_grid": (_i, [_vp, _i, _vp, _vp]),
    # learned initial density
    "cs_atom_descriptors": (_i, [_i, _dp, _i, _dp, _d, _dp]),
    "cs_atom_density": (_i, [_vp, _i, _dp, _i, _dp, _dp, _vp, _vp]),
    "cs_fit_workspace_bytes": (_i, [_vp, _i, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "cs_fit_atom_density": (_i, [_vp, _i, _dp, _i, _dp, _vp, _d, _dp, _vp, _vp]),
    "cs_mlp_create": (_i, [_i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_float), _i, _i,
                           ctypes.POINTER(_vp)]),
    "cs_mlp_free": (_i, [_vp]),
    "cs_mlp_param_count": (_i, [_vp, ctypes.POINTER(_ll)]),
    "cs_mlp_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "cs_mlp_forward": (_i, [_vp, _i, _vp, _vp, _vp]),
    "cs_mlp_loss_grad": (_i, [_vp, _i, _vp, _vp, ctypes.POINTER(ctypes.c_float),
                              ctypes.POINTER(ctypes.c_float), _vp]),
    "cs_mlp_train_step": (_i, [_vp, _i, _vp, _vp, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                               _vp]),
    "cs_mlp_last_error": (ctypes.c_char_p, [_vp]),
    "cs_scf_occupations": (_i, [_vp, _dp]),
    "cs_scf_free": (_i, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def library_path() -> str:
    return _LIB_PATH


def exported_symbols() -> list:
    return list(_SIGS)


class CsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


class Context:
    """Owns one cs_ctx (tables of a basis on a quadrature grid, bound to one device)."""

    def __init__(self, handle: int, device: int):
        self._h = ctypes.c_void_p(handle)
        self.device = device
        d = _ll()
        nr, nt, nph = _i(), _i(), _i()
        _lib.cs_basis_dims(self._h, ctypes.byref(d), ctypes.byref(nr), ctypes.byref(nt),
                           ctypes.byref(nph))
        self.d, self.n_r, self.n_theta, self.n_phi = d.value, nr.value, nt.value, nph.value
        self._ws = {}

    @property
    def handle(self):
        return self._h

    def check(self, status: int):
        if status != 0:
            raise CsError(status, _lib.cs_last_error(self._h).decode())

    def workspace(self, n_s: int, precision: int = CS_FP64) -> torch.Tensor:
        """A cached device workspace of cs_workspace_bytes(n_s, precision) bytes."""
        nbytes = cs_workspace_bytes(self, n_s, precision)
        key = (self.device,)
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.device}")
            self._ws[key] = ws
        return ws

    def close(self):
        if self._h is not None and self._h.value:
            _lib.cs_basis_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------- ABI mirrors
def cs_basis_init(R: float, lmax: int, nmax: int, n_r: int, n_theta: int, n_phi: int,
                  radial: int = CS_RADIAL_GAUSS_LEGENDRE, cuda_device: int = 0) -> Context:
    q = _Quad(n_r, n_theta, n_phi, radial)
    h = _vp()
    st = _lib.cs_basis_init(float(R), int(lmax), int(nmax), ctypes.byref(q), int(cuda_device),
                            ctypes.byref(h))
    if st != 0:
        raise CsError(st, _lib.cs_last_error(None).decode())
    return Context(h.value, cuda_device)


def cs_basis_free(ctx: Context):
    ctx.close()


def cs_basis_dims(ctx: Context):
    return ctx.d, ctx.n_r, ctx.n_theta, ctx.n_phi


def cs_grid(ctx: Context):
    """Host copies (numpy float64) of r, w_r, t, w_t, phi."""
    import numpy as np
    r, wr = np.empty(ctx.n_r), np.empty(ctx.n_r)
    t, wt = np.empty(ctx.n_theta), np.empty(ctx.n_theta)
    ph = np.empty(ctx.n_phi)
    c = lambda a: a.ctypes.data_as(_dp)  # noqa: E731
    ctx.check(_lib.cs_grid(ctx.handle, c(r), c(wr), c(t), c(wt), c(ph)))
    return r, wr, t, wt, ph


def cs_kinetic(ctx: Context):
    import numpy as np
    out = np.empty(ctx.d)
    ctx.check(_lib.cs_kinetic(ctx.handle, out.ctypes.data_as(_dp)))
    return out


def cs_bessel_zeros(ctx: Context, lmax: int, nmax: int):
    import numpy as np
    out = np.empty((lmax + 1) * nmax)
    ctx.check(_lib.cs_bessel_zeros(ctx.handle, out.ctypes.data_as(_dp)))
    return out.reshape(lmax + 1, nmax)


def cs_set_potential(ctx: Context, v_grid: torch.Tensor, stream=None):
    assert v_grid.dtype == torch.float64 and v_grid.is_cuda and v_grid.is_contiguous()
    assert v_grid.numel() == ctx.n_r * ctx.n_theta * ctx.n_phi
    ctx.check(_lib.cs_set_potential(ctx.handle, _ptr(v_grid), _stream_ptr(stream)))


def cs_set_projectors(ctx: Context, p_coef: torch.Tensor | None, h, stream=None):
    """p_coef: (n_p, d) float64 device tensor (rows = projector coefficient vectors)."""
    import numpy as np
    if p_coef is None or p_coef.shape[0] == 0:
        ctx.check(_lib.cs_set_projectors(ctx.handle, 0, None, None, _stream_ptr(stream)))
        return
    assert p_coef.dtype == torch.float64 and p_coef.is_contiguous() and p_coef.shape[1] == ctx.d
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    ctx.check(_lib.cs_set_projectors(ctx.handle, p_coef.shape[0], _ptr(p_coef),
                                     hh.ctypes.data_as(_dp), _stream_ptr(stream)))


def _check_block(ctx: Context, X: torch.Tensor, dtype):
    assert X.is_cuda and X.dtype == dtype and X.dim() == 2 and X.stride(1) == 1
    assert X.shape[1] >= ctx.d
    return X.shape[0], X.stride(0)


def cs_forward_transform(ctx: Context, g: torch.Tensor, coef: torch.Tensor, work=None,
                         stream=None):
    """g: (n, n_r, n_theta, n_phi) float64; coef: (n, ld) float64 (output)."""
    n, ld = _check_block(ctx, coef, torch.float64)
    assert g.is_contiguous() and g.dtype == torch.float64 and g.shape[0] == n
    work = ctx.workspace(n) if work is None else work
    ctx.check(_lib.cs_forward_transform(ctx.handle, n, _ptr(g), _ptr(coef), ld, _ptr(work),
                                        _stream_ptr(stream)))


def cs_inverse_transform(ctx: Context, coef: torch.Tensor, f: torch.Tensor, work=None,
                         stream=None):
    n, ld = _check_block(ctx, coef, torch.float64)
    assert f.is_contiguous() and f.dtype == torch.float64 and f.shape[0] == n
    work = ctx.workspace(n) if work is None else work
    ctx.check(_lib.cs_inverse_transform(ctx.handle, n, _ptr(coef), ld, _ptr(f), _ptr(work),
                                        _stream_ptr(stream)))


def cs_workspace_bytes(ctx: Context, n_s: int, precision: int = CS_FP64) -> int:
    out = ctypes.c_size_t()
    ctx.check(_lib.cs_workspace_bytes(ctx.handle, int(n_s), int(precision), ctypes.byref(out)))
    return out.value


def _dtype(precision):
    # FP64 and double-float blocks are double; FP32 and mixed blocks are float
    return torch.float64 if precision in (CS_FP64, CS_DF64) else torch.float32


def cs_apply_H(ctx: Context, X: torch.Tensor, HX: torch.Tensor, precision: int = CS_FP64,
               work=None, stream=None):
    n_s, ld = _check_block(ctx, X, _dtype(precision))
    assert HX.shape == X.shape and HX.stride() == X.stride() and HX.dtype == X.dtype
    work = ctx.workspace(n_s, precision) if work is None else work
    ctx.check(_lib.cs_apply_H(ctx.handle, n_s, _ptr(X), _ptr(HX), ld, int(precision),
                              _ptr(work), _stream_ptr(stream)))


def cs_apply_H_noalloc(ctx: Context, X: torch.Tensor, HX: torch.Tensor,
                       precision: int = CS_FP64, stream=None):
    """H X without a workspace, for callers that cannot allocate device memory at the call
    (another allocator holds the free memory, or cudaMalloc's synchronisation is not
    acceptable). Uses the library's built-in 32 MiB scratch; see include/cs.h for the
    size limit and the rule that overlapping calls on one device must be serialised."""
    n_s, ld = _check_block(ctx, X, _dtype(precision))
    assert HX.shape == X.shape and HX.stride() == X.stride() and HX.dtype == X.dtype
    ctx.check(_lib.cs_apply_H_noalloc(ctx.handle, n_s, _ptr(X), _ptr(HX), ld, int(precision),
                                      _stream_ptr(stream)))


def cs_cheb_filter(ctx: Context, X: torch.Tensor, degree: int, a: float, b: float, a0: float,
                   precision: int = CS_FP64, work=None, stream=None):
    n_s, ld = _check_block(ctx, X, _dtype(precision))
    work = ctx.workspace(n_s, precision) if work is None else work
    ctx.check(_lib.cs_cheb_filter(ctx.handle, n_s, _ptr(X), ld, int(degree), float(a),
                                  float(b), float(a0), int(precision), _ptr(work),
                                  _stream_ptr(stream)))


def cs_cholqr(ctx: Context, X: torch.Tensor, work=None, stream=None):
    n_s, ld = _check_block(ctx, X, torch.float64)
    work = ctx.workspace(n_s) if work is None else work
    ctx.check(_lib.cs_cholqr(ctx.handle, n_s, _ptr(X), ld, _ptr(work), _stream_ptr(stream)))


def cs_rayleigh_ritz(ctx: Context, X: torch.Tensor, theta: torch.Tensor, resid: torch.Tensor,
                     HX_out: torch.Tensor | None = None, work=None, stream=None):
    n_s, ld = _check_block(ctx, X, torch.float64)
    work = ctx.workspace(n_s) if work is None else work
    ctx.check(_lib.cs_rayleigh_ritz(ctx.handle, n_s, _ptr(X), ld, _ptr(theta), _ptr(resid),
                                    _ptr(HX_out), _ptr(work), _stream_ptr(stream)))


def cs_lanczos_bound(ctx: Context, v0: torch.Tensor, k: int = 10, work=None, stream=None):
    assert v0.is_cuda and v0.dtype == torch.float64 and v0.numel() >= ctx.d
    work = ctx.workspace(1) if work is None else work
    b, tmin = _d(), _d()
    ctx.check(_lib.cs_lanczos_bound(ctx.handle, int(k), _ptr(v0), ctypes.byref(b),
                                    ctypes.byref(tmin), _ptr(work), _stream_ptr(stream)))
    return b.value, tmin.value


def cs_chfsi(ctx: Context, X: torch.Tensor, n_want: int, degree: int, v0: torch.Tensor,
             theta: torch.Tensor, resid: torch.Tensor, tol: float = 1e-8, max_iter: int = 50,
             precision: int = CS_FP64, work=None, stream=None, raise_not_converged=True) -> int:
    n_s, ld = _check_block(ctx, X, torch.float64)
    work = ctx.workspace(n_s, precision) if work is None else work
    it = _i()
    st = _lib.cs_chfsi(ctx.handle, n_s, int(n_want), _ptr(X), ld, int(degree), float(tol),
                       int(max_iter), int(precision), _ptr(v0), _ptr(theta), _ptr(resid),
                       ctypes.byref(it), _ptr(work), _stream_ptr(stream))
    if st == 6 and not raise_not_converged:
        return it.value
    ctx.check(st)
    return it.value


def cs_chfsi_step(ctx: Context, X: torch.Tensor, degree: int, a: float, b: float, a0: float,
                  theta: torch.Tensor, resid: torch.Tensor, precision: int = CS_FP64,
                  work=None, stream=None):
    n_s, ld = _check_block(ctx, X, torch.float64)
    work = ctx.workspace(n_s, precision) if work is None else work
    ctx.check(_lib.cs_chfsi_step(ctx.handle, n_s, _ptr(X), ld, int(degree), float(a), float(b),
                                 float(a0), int(precision), _ptr(theta), _ptr(resid),
                                 _ptr(work), _stream_ptr(stream)))


def cs_cheb_filter_ritz(ctx: Context, X: torch.Tensor, HX: torch.Tensor, theta: torch.Tensor,
                        degree: int, a: float, b: float, a0: float, precision: int = CS_FP64,
                        work=None, stream=None):
    """p_m(H) X in residual form: X (FP64 Ritz vectors, filtered in place), HX = H X (FP64),
    theta = Ritz values (device, float64)."""
    n_s, ld = _check_block(ctx, X, torch.float64)
    _, ldh = _check_block(ctx, HX, torch.float64)
    assert HX.shape[0] == n_s and theta.is_cuda and theta.dtype == torch.float64
    work = ctx.workspace(n_s, precision) if work is None else work
    ctx.check(_lib.cs_cheb_filter_ritz(ctx.handle, n_s, _ptr(X), ld, _ptr(HX), ldh, _ptr(theta),
                                       int(degree), float(a), float(b), float(a0),
                                       int(precision), _ptr(work), _stream_ptr(stream)))


def cs_chfsi_step_ritz(ctx: Context, X: torch.Tensor, HX: torch.Tensor, degree: int, a: float,
                       b: float, a0: float, theta: torch.Tensor, resid: torch.Tensor,
                       precision: int = CS_FP64, work=None, stream=None):
    """One ChFSI iteration with the residual-form filter; X, HX, theta in/out."""
    n_s, ld = _check_block(ctx, X, torch.float64)
    assert HX.shape == X.shape and HX.stride() == X.stride() and HX.dtype == X.dtype
    work = ctx.workspace(n_s, precision) if work is None else work
    ctx.check(_lib.cs_chfsi_step_ritz(ctx.handle, n_s, _ptr(X), _ptr(HX), ld, int(degree),
                                      float(a), float(b), float(a0), int(precision),
                                      _ptr(theta), _ptr(resid), _ptr(work),
                                      _stream_ptr(stream)))


def cs_device_error(ctx: Context) -> int:
    """Reads and clears the context's device error word (0 = no bounded wait expired)."""
    code = _i()
    ctx.check(_lib.cs_device_error(ctx.handle, ctypes.byref(code)))
    return code.value


def cs_set_rr_precision(ctx: Context, precision: int):
    """Precision of the H X that Rayleigh-Ritz projects (default CS_FP64); the projection,
    eigensolve and residual norms stay FP64. Cached workspaces are re-sized on next use."""
    ctx.check(_lib.cs_set_rr_precision(ctx.handle, int(precision)))
    ctx._ws.clear()


def cs_set_dense_precision(ctx: Context, precision: int):
    """Arithmetic of the Cholesky-QR / Rayleigh-Ritz Gram matrices and block rotations:
    CS_FP64 (default), CS_DF64 (double-float on the FP32 pipe, FP64 storage) or CS_FP64_SLICED
    (exact integer-slice products on the tensor cores, rounded once)."""
    ctx.check(_lib.cs_set_dense_precision(ctx.handle, int(precision)))
    ctx._ws.clear()  # the workspace size depends on it


def cs_dense_gram(ctx: Context, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, work=None,
                  stream=None):
    """C = A^T B in the dense precision. A: (na, lda), B: (nb, ldb) float64 device blocks
    (rows = columns of the d x n matrices); C: (nb, ldc) float64, C[j, i] = (A^T B)[i, j]."""
    na, lda = _check_block(ctx, A, torch.float64)
    nb, ldb = _check_block(ctx, B, torch.float64)
    assert C.is_cuda and C.dtype == torch.float64 and C.stride(1) == 1 and C.shape[0] == nb
    assert C.shape[1] >= na
    work = ctx.workspace(max(na, nb)) if work is None else work
    ctx.check(_lib.cs_dense_gram(ctx.handle, na, nb, _ptr(A), lda, _ptr(B), ldb, _ptr(C),
                                 C.stride(0), _ptr(work), _stream_ptr(stream)))


def cs_dense_rotate(ctx: Context, A: torch.Tensor, Q: torch.Tensor, C: torch.Tensor, work=None,
                    stream=None):
    """C = A Q in the dense precision. A: (k, lda) float64 device block (d x k), Q: (n, ldq)
    float64 (the k x n matrix column by column), C: (n, ldc) (d x n)."""
    k, lda = _check_block(ctx, A, torch.float64)
    n, ldc = _check_block(ctx, C, torch.float64)
    assert Q.is_cuda and Q.dtype == torch.float64 and Q.stride(1) == 1 and Q.shape[0] == n
    assert Q.shape[1] >= k
    work = ctx.workspace(max(k, n)) if work is None else work
    ctx.check(_lib.cs_dense_rotate(ctx.handle, k, n, _ptr(A), lda, _ptr(Q), Q.stride(0),
                                   _ptr(C), ldc, _ptr(work), _stream_ptr(stream)))


def cs_profile_begin(ctx: Context):
    ctx.check(_lib.cs_profile_begin(ctx.handle))


PROFILE_FAMILIES = ("radial_synth", "angular", "radial_anal", "dense", "kb")
PROFILE_CLASSES = 3 * len(PROFILE_FAMILIES)


def profile_class_names():
    """Names of the profile classes: family (FP64 launches), family + '_f32' (FP32 / mixed),
    family + '_df64' (double-float)."""
    return (list(PROFILE_FAMILIES) + [f + "_f32" for f in PROFILE_FAMILIES] +
            [f + "_df64" for f in PROFILE_FAMILIES])


def cs_profile_end(ctx: Context):
    """Returns (ms, launches) per kernel class (profile_class_names())."""
    ms = (ctypes.c_double * PROFILE_CLASSES)()
    n = (_ll * PROFILE_CLASSES)()
    ctx.check(_lib.cs_profile_end(ctx.handle, ms, n))
    return list(ms), list(n)


class Batch:
    """Owns one cs_batch: many contexts filtered by one persistent launch per Chebyshev step."""

    def __init__(self, handle: int, ctxs, n_s, degree: int):
        self._h = ctypes.c_void_p(handle)
        self.ctxs = list(ctxs)  # keep the contexts alive
        self.n_s = list(n_s)
        self.degree = degree
        self._ws = None

    @property
    def handle(self):
        return self._h

    def check(self, status: int):
        if status != 0:
            raise CsError(status, _lib.cs_batch_last_error(self._h).decode())

    def workspace(self) -> torch.Tensor:
        if self._ws is None:
            self._ws = torch.empty(cs_batch_workspace_bytes(self), dtype=torch.uint8,
                                   device=f"cuda:{self.ctxs[0].device}")
        return self._ws

    def close(self):
        if self._h is not None and self._h.value:
            _lib.cs_batch_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cs_batch_create(ctxs, n_s, degree: int) -> Batch:
    n = len(ctxs)
    arr = (_vp * n)(*[c.handle.value for c in ctxs])
    ns = (_i * n)(*[int(x) for x in n_s])
    h = _vp()
    st = _lib.cs_batch_create(n, arr, ns, int(degree), ctypes.byref(h))
    if st != 0:
        raise CsError(st, "cs_batch_create failed (contexts must share a device, have a "
                          "potential and no projectors)")
    return Batch(h.value, ctxs, n_s, degree)


def cs_batch_free(batch: Batch):
    batch.close()


def cs_batch_workspace_bytes(batch: Batch) -> int:
    out = ctypes.c_size_t()
    batch.check(_lib.cs_batch_workspace_bytes(batch.handle, ctypes.byref(out)))
    return out.value


def _batch_args(batch: Batch, Xs, a, b, a0):
    import numpy as np
    n = len(batch.ctxs)
    assert len(Xs) == n
    for X, c in zip(Xs, batch.ctxs):
        assert X.is_cuda and X.dtype == torch.float32 and X.stride(1) == 1 and X.shape[1] >= c.d
    ptrs = (_vp * n)(*[X.data_ptr() for X in Xs])
    lds = (_ll * n)(*[X.stride(0) for X in Xs])
    av = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    bv = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    a0v = np.ascontiguousarray(np.asarray(a0, dtype=np.float64))
    return ptrs, lds, av, bv, a0v


def cs_batch_cheb_filter(batch: Batch, Xs, a, b, a0, work=None, stream=None):
    """Filters every block Xs[i] (float32, shape (n_s[i], ld)) in place with bounds
    (a[i], b[i], a0[i])."""
    ptrs, lds, av, bv, a0v = _batch_args(batch, Xs, a, b, a0)
    work = batch.workspace() if work is None else work
    batch.check(_lib.cs_batch_cheb_filter(batch.handle, ptrs, lds, av.ctypes.data_as(_dp),
                                          bv.ctypes.data_as(_dp), a0v.ctypes.data_as(_dp),
                                          _ptr(work), _stream_ptr(stream)))


def cs_batch_tune(batch: Batch, Xs, a, b, a0, work=None, stream=None):
    """Autotunes the angular tile variant on these blocks (restored afterwards); returns
    (variant, filter ms)."""
    ptrs, lds, av, bv, a0v = _batch_args(batch, Xs, a, b, a0)
    work = batch.workspace() if work is None else work
    ch = _i()
    ms = ctypes.c_float()
    batch.check(_lib.cs_batch_tune(batch.handle, ptrs, lds, av.ctypes.data_as(_dp),
                                   bv.ctypes.data_as(_dp), a0v.ctypes.data_as(_dp), _ptr(work),
                                   _stream_ptr(stream), ctypes.byref(ch), ctypes.byref(ms)))
    return ch.value, ms.value



BATCH_VARIANTS = ("persistent_rp4", "persistent_rp8", "persistent_rp2", "staged", "concurrent")


def cs_batch_set_variant(batch: Batch, variant):
    """Select a batch variant by index or by name (BATCH_VARIANTS)."""
    v = BATCH_VARIANTS.index(variant) if isinstance(variant, str) else int(variant)
    batch.check(_lib.cs_batch_set_variant(batch.handle, v))


def cs_batch_set_precision(batch: Batch, precision: int):
    """CS_FP32 (default) or CS_MIXED_BF16 (the concurrent variant only)."""
    batch.check(_lib.cs_batch_set_precision(batch.handle, int(precision)))


def cs_batch_tune_times(batch: Batch):
    """Filter time (ms) of each variant in the last tune (BATCH_VARIANTS order; -1: not run)."""
    ms = (ctypes.c_float * len(BATCH_VARIANTS))()
    batch.check(_lib.cs_batch_tune_times(batch.handle, ms, len(BATCH_VARIANTS)))
    return dict(zip(BATCH_VARIANTS, list(ms)))

def cs_batch_last_error(batch: Batch) -> str:
    return _lib.cs_batch_last_error(batch.handle).decode()


def cs_measure_peaks(cuda_device: int = 0):
    """(FP32, FP64) sustained fused multiply-add rates of the device in TFLOP/s."""
    f32, f64 = _d(), _d()
    st = _lib.cs_measure_peaks(int(cuda_device), ctypes.byref(f32), ctypes.byref(f64))
    if st != 0:
        raise CsError(st, "cs_measure_peaks failed")
    return f32.value, f64.value


def cs_last_error(ctx: Context | None) -> str:
    return _lib.cs_last_error(None if ctx is None else ctx.handle).decode()


def cs_launch_count(ctx: Context) -> int:
    return int(_lib.cs_launch_count(ctx.handle))


def grid_points(ctx: Context):
    """Cartesian coordinates (N_g, 3) of the context's quadrature grid in [k][j][q] order,
    for evaluating a potential or projector functions on it (host, numpy)."""
    import numpy as np
    r, _, t, _, ph = cs_grid(ctx)
    st = np.sqrt(1.0 - t * t)
    x = r[:, None, None] * st[None, :, None] * np.cos(ph)[None, None, :]
    y = r[:, None, None] * st[None, :, None] * np.sin(ph)[None, None, :]
    z = r[:, None, None] * t[None, :, None] * np.ones_like(ph)[None, None, :]
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def cs_lobpcg_workspace_bytes(ctx: Context, n_s: int) -> int:
    out = ctypes.c_size_t()
    ctx.check(_lib.cs_lobpcg_workspace_bytes(ctx.handle, int(n_s), ctypes.byref(out)))
    return out.value


def cs_lobpcg(ctx: Context, X: torch.Tensor, n_want: int, theta: torch.Tensor,
              resid: torch.Tensor, tol: float = 1e-8, max_iter: int = 200,
              precondition: bool = True, work=None, stream=None,
              raise_not_converged: bool = True):
    """LOBPCG with the Teter-Payne-Allan preconditioner; returns (iterations, restarts)."""
    n_s, ld = _check_block(ctx, X, torch.float64)
    if work is None:
        work = torch.empty(cs_lobpcg_workspace_bytes(ctx, n_s), dtype=torch.uint8,
                           device=f"cuda:{ctx.device}")
    it, rs = _i(), _i()
    st = _lib.cs_lobpcg(ctx.handle, n_s, int(n_want), _ptr(X), ld, float(tol), int(max_iter),
                        1 if precondition else 0, _ptr(theta), _ptr(resid), ctypes.byref(it),
                        ctypes.byref(rs), _ptr(work), _stream_ptr(stream))
    if st != 0 and not (st == 6 and not raise_not_converged):
        ctx.check(st)
    return it.value, rs.value


# ---------------------------------------------------------------------- SCF pieces
CS_DENSITY_CHUNK, CS_MIXER_MAX_HISTORY, CS_GRID_INTEGRALS_MAX = 16, 64, 8


def _check_grid(ctx: Context, t: torch.Tensor):
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    assert t.numel() == ctx.n_r * ctx.n_theta * ctx.n_phi


def cs_scf_workspace_bytes(ctx: Context) -> int:
    out = ctypes.c_size_t()
    ctx.check(_lib.cs_scf_workspace_bytes(ctx.handle, ctypes.byref(out)))
    return out.value


def _scf_ws(ctx: Context, work):
    if work is not None:
        return work
    nbytes = cs_scf_workspace_bytes(ctx)
    ws = ctx._ws.get("scf")
    if ws is None or ws.numel() < nbytes:
        ws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{ctx.device}")
        ctx._ws["scf"] = ws
    return ws


def cs_density(ctx: Context, X: torch.Tensor, occ: torch.Tensor, rho: torch.Tensor, work=None,
               stream=None):
    """rho = 2 sum_s occ[s] psi_s^2 on the grid (X: (n_s, ld) float64, occ: (n_s,) float64)."""
    n_s, ld = _check_block(ctx, X, torch.float64)
    assert occ.is_cuda and occ.dtype == torch.float64 and occ.numel() >= n_s
    _check_grid(ctx, rho)
    ctx.check(_lib.cs_density(ctx.handle, n_s, _ptr(X), ld, _ptr(occ), _ptr(rho),
                              _ptr(_scf_ws(ctx, work)), _stream_ptr(stream)))


def cs_hartree(ctx: Context, rho: torch.Tensor, vh: torch.Tensor, work=None, stream=None):
    _check_grid(ctx, rho)
    _check_grid(ctx, vh)
    ctx.check(_lib.cs_hartree(ctx.handle, _ptr(rho), _ptr(vh), _ptr(_scf_ws(ctx, work)),
                              _stream_ptr(stream)))


def cs_lda_xc(ctx: Context, rho: torch.Tensor, exc: torch.Tensor | None,
              vxc: torch.Tensor | None, stream=None):
    _check_grid(ctx, rho)
    for t in (exc, vxc):
        if t is not None:
            _check_grid(ctx, t)
    ctx.check(_lib.cs_lda_xc(ctx.handle, _ptr(rho), _ptr(exc), _ptr(vxc), _stream_ptr(stream)))


def cs_grid_integrals(ctx: Context, fs, gs=None, work=None, stream=None) -> list:
    """[sum_g W_g f_i g_i for i] (g_i None means 1)."""
    n = len(fs)
    gs = [None] * n if gs is None else list(gs)
    for t in list(fs) + [g for g in gs if g is not None]:
        _check_grid(ctx, t)
    fa = (_vp * n)(*[t.data_ptr() for t in fs])
    ga = (_vp * n)(*[None if g is None else g.data_ptr() for g in gs])
    out = (_d * n)()
    ctx.check(_lib.cs_grid_integrals(ctx.handle, n, fa, ga, out, _ptr(_scf_ws(ctx, work)),
                                     _stream_ptr(stream)))
    return list(out)


def cs_fermi_occupations(lam, n_electrons: float, kT: float):
    """(occ, mu, entropy) on the host (numpy)."""
    import numpy as np
    lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
    occ = np.empty_like(lam)
    mu, ent = _d(), _d()
    st = _lib.cs_fermi_occupations(lam.size, lam.ctypes.data_as(_dp), float(n_electrons),
                                   float(kT), occ.ctypes.data_as(_dp), ctypes.byref(mu),
                                   ctypes.byref(ent))
    if st != 0:
        raise CsError(st, "cs_fermi_occupations")
    return occ, mu.value, ent.value


class Mixer:
    """Owns one cs_mixer."""

    def __init__(self, ctx: Context, handle: int):
        self.ctx = ctx
        self._h = ctypes.c_void_p(handle)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h is not None and self._h.value:
            _lib.cs_mixer_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cs_mixer_create(ctx: Context, beta: float, history: int) -> Mixer:
    h = _vp()
    ctx.check(_lib.cs_mixer_create(ctx.handle, float(beta), int(history), ctypes.byref(h)))
    return Mixer(ctx, h.value)


def cs_mixer_mix(m: Mixer, x_in: torch.Tensor, x_out: torch.Tensor, x_next: torch.Tensor,
                 stream=None):
    for t in (x_in, x_out, x_next):
        _check_grid(m.ctx, t)
    m.ctx.check(_lib.cs_mixer_mix(m.handle, _ptr(x_in), _ptr(x_out), _ptr(x_next),
                                  _stream_ptr(stream)))


def cs_mixer_reset(m: Mixer):
    m.ctx.check(_lib.cs_mixer_reset(m.handle))


def cs_mixer_free(m: Mixer):
    m.close()


class Scf:
    """Owns one cs_scf."""

    def __init__(self, ctx: Context, handle: int, n_s: int):
        self.ctx = ctx
        self.n_s = n_s
        self._h = ctypes.c_void_p(handle)
        self._work = None

    @property
    def handle(self):
        return self._h

    def work(self) -> torch.Tensor:
        if self._work is None:
            self._work = torch.empty(cs_scf_work_bytes(self), dtype=torch.uint8,
                                     device=f"cuda:{self.ctx.device}")
        return self._work

    def close(self):
        if self._h is not None and self._h.value:
            _lib.cs_scf_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cs_scf_create(ctx: Context, params: ScfParams, v_ext: torch.Tensor, rho0: torch.Tensor,
                  v0: torch.Tensor) -> Scf:
    _check_grid(ctx, v_ext)
    _check_grid(ctx, rho0)
    assert v0.is_cuda and v0.dtype == torch.float64 and v0.numel() >= ctx.d
    h = _vp()
    ctx.check(_lib.cs_scf_create(ctx.handle, ctypes.byref(params), _ptr(v_ext), _ptr(rho0),
                                 _ptr(v0), ctypes.byref(h)))
    return Scf(ctx, h.value, params.n_s)


def cs_scf_work_bytes(s: Scf) -> int:
    out = ctypes.c_size_t()
    s.ctx.check(_lib.cs_scf_work_bytes(s.handle, ctypes.byref(out)))
    return out.value


def cs_scf_step(s: Scf, X: torch.Tensor, theta: torch.Tensor, resid: torch.Tensor, work=None,
                stream=None) -> dict:
    n_s, ld = _check_block(s.ctx, X, torch.float64)
    assert n_s == s.n_s
    rep = ScfReport()
    s.ctx.check(_lib.cs_scf_step(s.handle, _ptr(X), ld, _ptr(theta), _ptr(resid),
                                 _ptr(s.work() if work is None else work), _stream_ptr(stream),
                                 ctypes.byref(rep)))
    return rep.as_dict()


def cs_scf_grid(s: Scf, which: int, stream=None) -> torch.Tensor:
    """A copy (torch float64 (N_g,)) of one of the SCF state's grid functions: 0 v_in, 1 the
    last output density, 2 its Hartree potential, 3 its eps_xc, 4 v_ext."""
    ng = s.ctx.n_r * s.ctx.n_theta * s.ctx.n_phi
    out = torch.empty(ng, dtype=torch.float64, device=f"cuda:{s.ctx.device}")
    s.ctx.check(_lib.cs_scf_grid(s.handle, int(which), _ptr(out), _stream_ptr(stream)))
    return out


def cs_scf_occupations(s: Scf):
    import numpy as np
    out = np.empty(s.n_s)
    s.ctx.check(_lib.cs_scf_occupations(s.handle, out.ctypes.data_as(_dp)))
    return out


def cs_scf_free(s: Scf):
    s.close()


# ---------------------------------------------------------------------- learned density
def cs_atom_descriptors(atoms, mu, width: float):
    """(n_atoms, len(mu)) numpy descriptors of the atoms (n_atoms, 3)."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64))
    m = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    out = np.empty((a.shape[0], m.size))
    st = _lib.cs_atom_descriptors(a.shape[0], a.ctypes.data_as(_dp), m.size,
                                  m.ctypes.data_as(_dp), float(width), out.ctypes.data_as(_dp))
    if st != 0:
        raise CsError(st, "cs_atom_descriptors")
    return out


def cs_atom_density(ctx: Context, atoms, sigmas, coef, rho: torch.Tensor, stream=None):
    """rho += sum_a sum_j coef[a, j] phi_j(|x - a|) (rho: device float64 grid)."""
    import numpy as np
    _check_grid(ctx, rho)
    a = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64))
    sg = np.ascontiguousarray(np.asarray(sigmas, dtype=np.float64))
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
    ctx.check(_lib.cs_atom_density(ctx.handle, a.shape[0], a.ctypes.data_as(_dp), sg.size,
                                   sg.ctypes.data_as(_dp), c.ctypes.data_as(_dp), _ptr(rho),
                                   _stream_ptr(stream)))


def cs_fit_workspace_bytes(ctx: Context, n_atoms: int, n_basis: int) -> int:
    out = ctypes.c_size_t()
    ctx.check(_lib.cs_fit_workspace_bytes(ctx.handle, int(n_atoms), int(n_basis), ctypes.byref(out)))
    return out.value


def cs_fit_atom_density(ctx: Context, atoms, sigmas, target: torch.Tensor, ridge: float = 1e-10,
                        work=None, stream=None):
    """Least-squares coefficients (n_atoms, n_basis) of the atom-centred expansion of target."""
    import numpy as np
    _check_grid(ctx, target)
    a = np.ascontiguousarray(np.asarray(atoms, dtype=np.float64))
    sg = np.ascontiguousarray(np.asarray(sigmas, dtype=np.float64))
    out = np.empty((a.shape[0], sg.size))
    if work is None:
        work = torch.empty(cs_fit_workspace_bytes(ctx, a.shape[0], sg.size), dtype=torch.uint8,
                           device=f"cuda:{ctx.device}")
    ctx.check(_lib.cs_fit_atom_density(ctx.handle, a.shape[0], a.ctypes.data_as(_dp), sg.size,
                                       sg.ctypes.data_as(_dp), _ptr(target), float(ridge),
                                       out.ctypes.data_as(_dp), _ptr(work), _stream_ptr(stream)))
    return out


class Mlp:
    """Owns one cs_mlp. Activations are float32 column-major (n rows = atoms): pass torch
    tensors of shape (features, n) (C order), i.e. row f holds feature f of every atom."""

    def __init__(self, handle: int, dims):
        self._h = ctypes.c_void_p(handle)
        self.dims = list(dims)

    @property
    def handle(self):
        return self._h

    def check(self, status: int):
        if status != 0:
            raise CsError(status, _lib.cs_mlp_last_error(self._h).decode())

    def close(self):
        if self._h is not None and self._h.value:
            _lib.cs_mlp_free(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cs_mlp_create(dims, params, max_rows: int, cuda_device: int = 0) -> Mlp:
    """params: flat float32 (W_1 column-major n_in x n_out, b_1, W_2, b_2, ...)."""
    import numpy as np
    d = (_i * len(dims))(*[int(x) for x in dims])
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    h = _vp()
    st = _lib.cs_mlp_create(len(dims) - 1, d, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                            int(max_rows), int(cuda_device), ctypes.byref(h))
    if st != 0:
        raise CsError(st, "cs_mlp_create")
    return Mlp(h.value, dims)


def cs_mlp_free(m: Mlp):
    m.close()


def cs_mlp_param_count(m: Mlp) -> int:
    c = _ll()
    m.check(_lib.cs_mlp_param_count(m.handle, ctypes.byref(c)))
    return c.value


def cs_mlp_params(m: Mlp):
    import numpy as np
    out = np.empty(cs_mlp_param_count(m), dtype=np.float32)
    m.check(_lib.cs_mlp_params(m.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def _check_act(t: torch.Tensor, rows: int):
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.shape[0] == rows


def cs_mlp_forward(m: Mlp, X: torch.Tensor, stream=None) -> torch.Tensor:
    _check_act(X, m.dims[0])
    n = X.shape[1]
    Y = torch.empty((m.dims[-1], n), dtype=torch.float32, device=X.device)
    m.check(_lib.cs_mlp_forward(m.handle, n, _ptr(X), _ptr(Y), _stream_ptr(stream)))
    return Y


def cs_mlp_loss_grad(m: Mlp, X: torch.Tensor, T: torch.Tensor, stream=None):
    import numpy as np
    _check_act(X, m.dims[0])
    _check_act(T, m.dims[-1])
    loss = ctypes.c_float()
    g = np.empty(cs_mlp_param_count(m), dtype=np.float32)
    m.check(_lib.cs_mlp_loss_grad(m.handle, X.shape[1], _ptr(X), _ptr(T), ctypes.byref(loss),
                                  g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                  _stream_ptr(stream)))
    return loss.value, g


def cs_mlp_train_step(m: Mlp, X: torch.Tensor, T: torch.Tensor, lr: float, want_loss=True,
                      stream=None):
    _check_act(X, m.dims[0])
    _check_act(T, m.dims[-1])
    loss = ctypes.c_float()
    m.check(_lib.cs_mlp_train_step(m.handle, X.shape[1], _ptr(X), _ptr(T), float(lr),
                                   ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)))
    return loss.value if want_loss else None


def cs_mlp_last_error(m: Mlp) -> str:
    return _lib.cs_mlp_last_error(m.handle).decode()
