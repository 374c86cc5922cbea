"""ctypes binding of the C ABI in include/helm.h (argument marshalling only).

Every numerical step runs in libhelm.so's CUDA kernels; this module only
checks tensor types, hands device pointers and the current CUDA stream to
the library and allocates the caller-owned workspace with torch.  Importing
it loads the library and raises if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# HELM_LIBRARY=debug selects the bounds-checking build (libhelm_debug.so)
LIB_PATH = os.path.join(_HERE, "libhelm_debug.so" if os.environ.get("HELM_LIBRARY") == "debug" else "libhelm.so")

HELM_OK, HELM_E_INVAL, HELM_E_NOMEM, HELM_E_CUDA, HELM_E_NOCONV, HELM_E_NONFINITE, HELM_E_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6
HELM_E_BOUNDS = -7  # debug build only
FP64, MIXED = 0, 1
FIELD_C128, FIELD_C64 = 0, 1
PRECOND_NONE, PRECOND_JACOBI, PRECOND_MLGMRES = 0, 1, 2
CALL_APPLY, CALL_FORWARD, CALL_ADJOINT, CALL_MISFIT_GRAD, CALL_MISFIT, CALL_GRADIENT, CALL_PRECOND = \
    0, 1, 2, 3, 4, 5, 6
CALL_BORN, CALL_BORN_ADJOINT, CALL_GN_HESSVEC, CALL_HESSVEC, CALL_MISFIT_GRAD_25D, CALL_WRI = 7, 8, 9, 10, 11, 12
PROF_CLASSES = ["stencil_c64", "stencil_c128", "krylov_c64", "krylov_c128", "small", "transfer", "fwi",
                "misc", "stencil_c64_coarse", "krylov_c64_coarse", "gram_c64", "update_c64"]


class HelmGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("npml", ctypes.c_int * 3), ("v_ref", ctypes.c_double),
                ("sigma_max", ctypes.c_double * 3), ("levels", ctypes.c_int)]


class HelmSolveOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("precond", ctypes.c_int), ("k_inner", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("tol", ctypes.c_double), ("tol_inner", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("k_so", ctypes.c_int), ("k_si", ctypes.c_int),
                ("k_co", ctypes.c_int), ("k_ci", ctypes.c_int), ("jacobi_omega", ctypes.c_double),
                ("jacobi_sweeps", ctypes.c_int), ("max_batch", ctypes.c_int), ("reorth", ctypes.c_int),
                ("sstep", ctypes.c_int)]


class HelmRhsReport(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_resid", ctypes.c_double)]


class HelmBatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("m_phys", ctypes.c_void_p), ("freqs_hz", ctypes.POINTER(ctypes.c_double)),
                ("nfreq", ctypes.c_int), ("src_idx", ctypes.c_void_p), ("n_srcloc", ctypes.c_int),
                ("Q", ctypes.c_void_p), ("nsrc", ctypes.c_int), ("wavelet", ctypes.c_void_p),
                ("rec_idx", ctypes.c_void_p), ("nrec", ctypes.c_int), ("d_obs", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("f_out", ctypes.c_void_p), ("g_out", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t),
                ("reports", ctypes.POINTER(HelmRhsReport)), ("stream", ctypes.c_void_p), ("status", ctypes.c_int)]


EXPORTS = ["helm_default_opts", "helm_misfit_and_gradient_batch", "helm_plan_create", "helm_plan_destroy", "helm_plan_dims",
           "helm_workspace_size", "helm_apply", "helm_precond_apply", "helm_forward", "helm_adjoint", "misfit_and_gradient",
           "helm_misfit", "helm_gradient", "helm_born", "helm_born_adjoint", "helm_gn_hessvec", "helm_hessvec",
           "helm_misfit_and_gradient_25d", "helm_wri_misfit_and_gradient",
           "helm_status_string", "helm_kernel_launch_count", "helm_profile_enable", "helm_profile_read",
           "helm_check_bounded_wait", "helm_stencil_variant_count", "helm_stencil_variant_info",
           "helm_stencil_select", "helm_stencil_tuned"]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libhelm.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    lib.helm_default_opts.argtypes = [ctypes.POINTER(HelmSolveOpts)]
    lib.helm_plan_create.argtypes = [ctypes.POINTER(HelmGrid), ctypes.POINTER(HelmSolveOpts),
                                     ctypes.POINTER(ctypes.c_void_p)]
    lib.helm_plan_destroy.argtypes = [P]
    lib.helm_plan_destroy.restype = None
    lib.helm_plan_dims.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(S), ctypes.POINTER(S)]
    lib.helm_workspace_size.argtypes = [P, I, I, I, I, ctypes.POINTER(S)]
    lib.helm_apply.argtypes = [P, P, D, I, I, P, P, I, P, S, P]
    lib.helm_precond_apply.argtypes = [P, P, D, I, P, P, I, P, S, P]
    lib.helm_forward.argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, P, I, P, P, P, P, S,
                                 ctypes.POINTER(HelmRhsReport), P]
    lib.helm_adjoint.argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, P, S,
                                 ctypes.POINTER(HelmRhsReport), P]
    lib.misfit_and_gradient.argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, P, I, P, P, P, P, P, S,
                                        ctypes.POINTER(HelmRhsReport), P]
    for name in ("helm_born", "helm_born_adjoint", "helm_gn_hessvec"):
        getattr(lib, name).argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, P, I, P, P, P, P, S,
                                       ctypes.POINTER(HelmRhsReport), P]
    lib.helm_hessvec.argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, P, I, P, P, P, P, P, S,
                                 ctypes.POINTER(HelmRhsReport), P]
    lib.helm_misfit_and_gradient_25d.argtypes = [P, P, ctypes.POINTER(D), I, ctypes.POINTER(D), ctypes.POINTER(D), I,
                                                 P, I, P, I, P, P, I, P, P, P, P, S, ctypes.POINTER(HelmRhsReport), P]
    lib.helm_wri_misfit_and_gradient.argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, P, I, P, D, D, I, P, P, P,
                                                 S, ctypes.POINTER(HelmRhsReport), P]
    lib.helm_misfit.argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, P, I, P, P, P, P, P, I, P, S,
                                ctypes.POINTER(HelmRhsReport), P]
    lib.helm_gradient.argtypes = [P, P, ctypes.POINTER(D), I, P, I, P, I, P, I, P, P, P, S,
                                  ctypes.POINTER(HelmRhsReport), P]
    lib.helm_misfit_and_gradient_batch.argtypes = [ctypes.POINTER(HelmBatchItem), I, I]
    lib.helm_check_bounded_wait.argtypes = [P]
    lib.helm_stencil_variant_count.argtypes = []
    lib.helm_stencil_variant_info.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.helm_stencil_select.argtypes = [I]
    lib.helm_stencil_tuned.argtypes = [P, I, I, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.helm_status_string.argtypes = [I]
    lib.helm_status_string.restype = ctypes.c_char_p
    lib.helm_kernel_launch_count.argtypes = []
    lib.helm_kernel_launch_count.restype = ctypes.c_uint64
    lib.helm_profile_enable.argtypes = [I]
    lib.helm_profile_read.argtypes = [I, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(D),
                                      ctypes.POINTER(D)]
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class HelmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {lib().helm_status_string(code).decode()} ({code})")


def _check(code: int, where: str, allow_noconv: bool = False):
    if code == HELM_OK or (allow_noconv and code == HELM_E_NOCONV):
        return code
    raise HelmError(code, where)


def default_opts(**kw) -> HelmSolveOpts:
    o = HelmSolveOpts()
    lib().helm_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def make_grid(dim: int, n: Sequence[int], h: float, npml: Sequence[int], v_ref: float,
              levels: int = 1, sigma_max: Sequence[float] = (0.0, 0.0, 0.0)) -> HelmGrid:
    g = HelmGrid()
    g.dim = dim
    g.n[:] = list(n)
    g.h = h
    g.npml[:] = list(npml)
    g.v_ref = v_ref
    g.sigma_max[:] = list(sigma_max)
    g.levels = levels
    return g


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Plan:
    """A helm_plan plus a cached caller-owned workspace."""

    def __init__(self, grid: HelmGrid, opts: Optional[HelmSolveOpts] = None, device="cuda"):
        self.grid = grid
        self.opts = opts if opts is not None else default_opts()
        self.device = torch.device(device)
        h = ctypes.c_void_p()
        _check(lib().helm_plan_create(ctypes.byref(grid), ctypes.byref(self.opts), ctypes.byref(h)),
               "helm_plan_create")
        self._h = h
        N = (ctypes.c_int * 3)()
        nc, nph = ctypes.c_size_t(), ctypes.c_size_t()
        lib().helm_plan_dims(h, N, ctypes.byref(nc), ctypes.byref(nph))
        self.N = tuple(N)
        self.n_comp = nc.value
        self.n_phys = nph.value
        self._ws: Optional[torch.Tensor] = None

    def close(self):
        if getattr(self, "_h", None):
            lib().helm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def comp_shape(self):
        return (self.N[2], self.N[1], self.N[0])

    def workspace_size(self, call: int, nfreq: int, nsrc: int, nrec: int) -> int:
        b = ctypes.c_size_t()
        _check(lib().helm_workspace_size(self._h, call, nfreq, nsrc, nrec, ctypes.byref(b)),
               "helm_workspace_size")
        return b.value

    def workspace(self, nbytes: int):
        """Device scratch of at least nbytes, 256-byte aligned (grown on demand)."""
        if self._ws is None or self._ws.numel() < nbytes + 256:
            self._ws = None
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        p = self._ws.data_ptr()
        off = (-p) % 256
        return ctypes.c_void_p(p + off), self._ws.numel() - off


def _need(cond: bool, msg: str):
    if not cond:
        raise ValueError(msg)


def _check_common(plan: "Plan", m_phys, src_idx=None, Q=None, wavelet=None, nfreq=None):
    _need(m_phys.numel() == plan.n_phys, f"m_phys must hold n_phys={plan.n_phys} values")
    if Q is not None:
        _need(Q.dim() == 2 and Q.shape[0] == src_idx.numel(), "Q must be [n_srcloc, nsrc]")
    if wavelet is not None:
        _need(wavelet.numel() == nfreq, "wavelet must hold one value per frequency")


def _freqs(freqs_hz) -> ctypes.Array:
    f = np.ascontiguousarray(np.asarray(freqs_hz, dtype=np.float64).ravel())
    return (ctypes.c_double * len(f))(*f.tolist())


def helm_apply(plan: Plan, m_phys: torch.Tensor, freq_hz: float, x: torch.Tensor, adjoint: bool = False,
               out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """y = H x (or H^H x) for x of shape (nrhs, n_comp) complex128 (FP64) or complex64."""
    _dev(m_phys, torch.float64, "m_phys")
    _check_common(plan, m_phys)
    if x.dtype == torch.complex128:
        prec = FP64
    elif x.dtype == torch.complex64:
        prec = MIXED
    else:
        raise TypeError("x must be complex128 or complex64")
    _dev(x, x.dtype, "x")
    nrhs = x.numel() // plan.n_comp
    if nrhs * plan.n_comp != x.numel():
        raise ValueError("x must hold whole fields")
    y = torch.empty_like(x) if out is None else out
    _need(y.dtype == x.dtype and y.numel() == x.numel() and y.is_contiguous() and y.data_ptr() != x.data_ptr(),
          "out must be a distinct contiguous tensor like x")
    ws, nb = plan.workspace(plan.workspace_size(CALL_APPLY, 1, nrhs, 0))
    _check(lib().helm_apply(plan._h, _ptr(m_phys), float(freq_hz), int(bool(adjoint)), prec, _ptr(x),
                            _ptr(y), nrhs, ws, nb, _stream(x.device)), "helm_apply")
    return y


def helm_precond_apply(plan: Plan, m_phys: torch.Tensor, freq_hz: float, x: torch.Tensor, adjoint: bool = False,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """z = M^{-1} x (one V-cycle, Jacobi sweeps or a copy, as the plan's options
    say) for x of shape (nrhs, n_comp): complex128 for an FP64 plan, complex64
    for a mixed-precision plan."""
    _dev(m_phys, torch.float64, "m_phys")
    _check_common(plan, m_phys)
    want = torch.complex128 if plan.opts.precision == FP64 else torch.complex64
    _need(x.dtype == want, f"x must be {want} for this plan's precision")
    _dev(x, x.dtype, "x")
    nrhs = x.numel() // plan.n_comp
    if nrhs * plan.n_comp != x.numel():
        raise ValueError("x must hold whole fields")
    z = torch.empty_like(x) if out is None else out
    _need(z.dtype == x.dtype and z.numel() == x.numel() and z.is_contiguous() and z.data_ptr() != x.data_ptr(),
          "out must be a distinct contiguous tensor like x")
    ws, nb = plan.workspace(plan.workspace_size(CALL_PRECOND, 1, nrhs, 0))
    _check(lib().helm_precond_apply(plan._h, _ptr(m_phys), float(freq_hz), int(bool(adjoint)), _ptr(x), _ptr(z),
                                    nrhs, ws, nb, _stream(x.device)), "helm_precond_apply")
    return z


def stencil_variants() -> list:
    """Tile shapes of the complex64 operator apply: dicts of threads, zplanes, min_blocks."""
    out = []
    for v in range(int(lib().helm_stencil_variant_count())):
        t, z, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().helm_stencil_variant_info(v, ctypes.byref(t), ctypes.byref(z), ctypes.byref(b)),
               "helm_stencil_variant_info")
        out.append(dict(threads=t.value, zplanes=z.value, min_blocks=b.value))
    return out


def stencil_select(variant: int):
    """Force tile shape `variant` for every later apply (-1: tune per grid on first use)."""
    _check(lib().helm_stencil_select(int(variant)), "helm_stencil_select")


def stencil_tuned(plan: "Plan", level: int = 0, residual: bool = False):
    """(shape, microseconds) tuned for the plan's grid level, or None when not tuned yet."""
    v, us = ctypes.c_int(), ctypes.c_double()
    code = lib().helm_stencil_tuned(plan._h, int(level), int(bool(residual)), ctypes.byref(v), ctypes.byref(us))
    return (v.value, us.value) if code == HELM_OK else None


def check_bounded_wait(device="cuda") -> int:
    """Status of the library's bounded-wait self-check (HELM_E_TIMEOUT expected)."""
    return int(lib().helm_check_bounded_wait(_stream(torch.device(device))))


def _reports(n):
    return (HelmRhsReport * n)()


def reports_to_list(rep):
    return [dict(status=r.status, iters=r.iters, refinements=r.refinements, rel_resid=r.rel_resid)
            for r in rep]


def helm_forward(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, wavelet=None, want_fields=True,
                 want_data=True, U0=None):
    """Returns (U [nfreq, nsrc, n_comp] or None, D [nfreq, nsrc, nrec] or None, reports).
    U0 (complex128 [nfreq, nsrc, n_comp]) warm-starts the solves."""
    _dev(m_phys, torch.float64, "m_phys")
    _dev(src_idx, torch.int32, "src_idx")
    _dev(Q, torch.complex128, "Q")
    _dev(rec_idx, torch.int32, "rec_idx")
    if wavelet is not None:
        _dev(wavelet, torch.complex128, "wavelet")
    nfreq = len(np.atleast_1d(freqs_hz))
    _check_common(plan, m_phys, src_idx, Q, wavelet, nfreq)
    nsrc = Q.shape[1]
    nrec = rec_idx.numel()
    dev = m_phys.device
    if U0 is not None:
        _dev(U0, torch.complex128, "U0")
        _need(tuple(U0.shape) == (nfreq, nsrc, plan.n_comp), "U0 must be [nfreq, nsrc, n_comp]")
    U = torch.empty((nfreq, nsrc, plan.n_comp), dtype=torch.complex128, device=dev) if want_fields else None
    D = torch.empty((nfreq, nsrc, nrec), dtype=torch.complex128, device=dev) if want_data else None
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(CALL_FORWARD, nfreq, nsrc, nrec))
    code = lib().helm_forward(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(src_idx), src_idx.numel(),
                              _ptr(Q), nsrc, _ptr(wavelet), _ptr(rec_idx), nrec, _ptr(U0), _ptr(U), _ptr(D), ws, nb,
                              rep, _stream(dev))
    _check(code, "helm_forward", allow_noconv=True)
    return U, D, reports_to_list(rep)


def helm_adjoint(plan: Plan, m_phys, freqs_hz, rec_idx, R_in):
    """V = H^{-H} P_r^T R for R_in [nfreq, nsrc, nrec]; returns (V, reports)."""
    _dev(m_phys, torch.float64, "m_phys")
    _dev(rec_idx, torch.int32, "rec_idx")
    _dev(R_in, torch.complex128, "R_in")
    _check_common(plan, m_phys)
    _need(R_in.dim() == 3 and R_in.shape[0] == len(np.atleast_1d(freqs_hz)) and R_in.shape[2] == rec_idx.numel(),
          "R_in must be [nfreq, nsrc, nrec]")
    nfreq, nsrc, nrec = R_in.shape
    V = torch.empty((nfreq, nsrc, plan.n_comp), dtype=torch.complex128, device=m_phys.device)
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(CALL_ADJOINT, nfreq, nsrc, nrec))
    code = lib().helm_adjoint(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(rec_idx), nrec, _ptr(R_in),
                              nsrc, _ptr(V), ws, nb, rep, _stream(m_phys.device))
    _check(code, "helm_adjoint", allow_noconv=True)
    return V, reports_to_list(rep)


def misfit_and_gradient(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, wavelet=None, mask=None,
                        f_out=None, g_out=None):
    """Returns (f [1] float64, g [n_phys] float64, reports); all device tensors."""
    _dev(m_phys, torch.float64, "m_phys")
    _dev(src_idx, torch.int32, "src_idx")
    _dev(Q, torch.complex128, "Q")
    _dev(rec_idx, torch.int32, "rec_idx")
    _dev(d_obs, torch.complex128, "d_obs")
    if wavelet is not None:
        _dev(wavelet, torch.complex128, "wavelet")
    if mask is not None:
        _dev(mask, torch.uint8, "mask")
    nfreq = len(np.atleast_1d(freqs_hz))
    _check_common(plan, m_phys, src_idx, Q, wavelet, nfreq)
    nsrc = Q.shape[1]
    nrec = rec_idx.numel()
    _need(tuple(d_obs.shape) == (nfreq, nsrc, nrec), "d_obs must be [nfreq, nsrc, nrec]")
    if mask is not None:
        _need(mask.numel() == nfreq * nsrc, "mask must be [nfreq, nsrc]")
    dev = m_phys.device
    f = torch.empty(1, dtype=torch.float64, device=dev) if f_out is None else f_out
    g = torch.empty(plan.n_phys, dtype=torch.float64, device=dev) if g_out is None else g_out
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(CALL_MISFIT_GRAD, nfreq, nsrc, nrec))
    code = lib().misfit_and_gradient(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(src_idx),
                                     src_idx.numel(), _ptr(Q), nsrc, _ptr(wavelet), _ptr(rec_idx), nrec,
                                     _ptr(d_obs), _ptr(mask), _ptr(f), _ptr(g), ws, nb, rep, _stream(dev))
    _check(code, "misfit_and_gradient", allow_noconv=True)
    return f, g, reports_to_list(rep)


def _linearised(name, call, plan, m_phys, freqs_hz, src_idx, Q, rec_idx, vec, wavelet, mask):
    _dev(m_phys, torch.float64, "m_phys")
    _dev(src_idx, torch.int32, "src_idx")
    _dev(Q, torch.complex128, "Q")
    _dev(rec_idx, torch.int32, "rec_idx")
    if wavelet is not None:
        _dev(wavelet, torch.complex128, "wavelet")
    if mask is not None:
        _dev(mask, torch.uint8, "mask")
    nfreq = len(np.atleast_1d(freqs_hz))
    _check_common(plan, m_phys, src_idx, Q, wavelet, nfreq)
    nsrc, nrec = Q.shape[1], rec_idx.numel()
    if mask is not None:
        _need(mask.numel() == nfreq * nsrc, "mask must be [nfreq, nsrc]")
    dev = m_phys.device
    if call == CALL_BORN_ADJOINT:
        _dev(vec, torch.complex128, "dD")
        _need(tuple(vec.shape) == (nfreq, nsrc, nrec), "dD must be [nfreq, nsrc, nrec]")
    else:
        _dev(vec, torch.float64, "dm_phys")
        _need(vec.numel() == plan.n_phys, f"dm_phys must hold n_phys={plan.n_phys} values")
    if call == CALL_BORN:
        out = torch.empty((nfreq, nsrc, nrec), dtype=torch.complex128, device=dev)
    else:
        out = torch.empty(plan.n_phys, dtype=torch.float64, device=dev)
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(call, nfreq, nsrc, nrec))
    code = getattr(lib(), name)(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(src_idx), src_idx.numel(),
                                _ptr(Q), nsrc, _ptr(wavelet), _ptr(rec_idx), nrec, _ptr(vec), _ptr(mask), _ptr(out),
                                ws, nb, rep, _stream(dev))
    _check(code, name, allow_noconv=True)
    return out, reports_to_list(rep)


def helm_born(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, dm_phys, wavelet=None, mask=None):
    """dD = J dm [nfreq, nsrc, nrec] complex128 (two solves per pair); returns (dD, reports)."""
    return _linearised("helm_born", CALL_BORN, plan, m_phys, freqs_hz, src_idx, Q, rec_idx, dm_phys, wavelet, mask)


def helm_born_adjoint(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, dD, wavelet=None, mask=None):
    """g = J^T dD [n_phys] float64 (two solves per pair); returns (g, reports)."""
    return _linearised("helm_born_adjoint", CALL_BORN_ADJOINT, plan, m_phys, freqs_hz, src_idx, Q, rec_idx, dD,
                       wavelet, mask)


def helm_gn_hessvec(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, dm_phys, wavelet=None, mask=None):
    """J^T J dm [n_phys] float64 (three solves per pair); returns (Hdm, reports)."""
    return _linearised("helm_gn_hessvec", CALL_GN_HESSVEC, plan, m_phys, freqs_hz, src_idx, Q, rec_idx, dm_phys,
                       wavelet, mask)


def helm_hessvec(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, dm_phys, wavelet=None, mask=None):
    """Full Hessian of the misfit times dm, [n_phys] float64 (four solves per pair);
    returns (Hdm, reports)."""
    _dev(m_phys, torch.float64, "m_phys")
    _dev(src_idx, torch.int32, "src_idx")
    _dev(Q, torch.complex128, "Q")
    _dev(rec_idx, torch.int32, "rec_idx")
    _dev(d_obs, torch.complex128, "d_obs")
    _dev(dm_phys, torch.float64, "dm_phys")
    if wavelet is not None:
        _dev(wavelet, torch.complex128, "wavelet")
    if mask is not None:
        _dev(mask, torch.uint8, "mask")
    nfreq = len(np.atleast_1d(freqs_hz))
    _check_common(plan, m_phys, src_idx, Q, wavelet, nfreq)
    nsrc, nrec = Q.shape[1], rec_idx.numel()
    _need(tuple(d_obs.shape) == (nfreq, nsrc, nrec), "d_obs must be [nfreq, nsrc, nrec]")
    _need(dm_phys.numel() == plan.n_phys, f"dm_phys must hold n_phys={plan.n_phys} values")
    if mask is not None:
        _need(mask.numel() == nfreq * nsrc, "mask must be [nfreq, nsrc]")
    dev = m_phys.device
    out = torch.empty(plan.n_phys, dtype=torch.float64, device=dev)
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(CALL_HESSVEC, nfreq, nsrc, nrec))
    code = lib().helm_hessvec(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(src_idx), src_idx.numel(), _ptr(Q),
                              nsrc, _ptr(wavelet), _ptr(rec_idx), nrec, _ptr(d_obs), _ptr(dm_phys), _ptr(mask),
                              _ptr(out), ws, nb, rep, _stream(dev))
    _check(code, "helm_hessvec", allow_noconv=True)
    return out, reports_to_list(rep)


def misfit_and_gradient_25d(plan: Plan, m_phys, freqs_hz, ky, ck, src_idx, Q, rec_idx, d_obs, wavelet=None):
    """2.5D misfit and gradient on a 2D plan: data = sum_i ck[i] P_r u~_i over the
    wavenumbers ky (host arrays).  Returns (f [1], g [n_phys], reports [nfreq*nsrc*nk])."""
    _need(plan.grid.dim == 2, "2.5D needs a 2D plan")
    _dev(m_phys, torch.float64, "m_phys")
    _dev(src_idx, torch.int32, "src_idx")
    _dev(Q, torch.complex128, "Q")
    _dev(rec_idx, torch.int32, "rec_idx")
    _dev(d_obs, torch.complex128, "d_obs")
    if wavelet is not None:
        _dev(wavelet, torch.complex128, "wavelet")
    nfreq = len(np.atleast_1d(freqs_hz))
    _check_common(plan, m_phys, src_idx, Q, wavelet, nfreq)
    ky = np.ascontiguousarray(np.asarray(ky, dtype=np.float64).ravel())
    ck = np.ascontiguousarray(np.asarray(ck, dtype=np.float64).ravel())
    _need(ky.size == ck.size and ky.size >= 1, "ky and ck must have the same length >= 1")
    nk, nsrc, nrec = ky.size, Q.shape[1], rec_idx.numel()
    _need(tuple(d_obs.shape) == (nfreq, nsrc, nrec), "d_obs must be [nfreq, nsrc, nrec]")
    dev = m_phys.device
    f = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(plan.n_phys, dtype=torch.float64, device=dev)
    rep = _reports(nfreq * nsrc * nk)
    ws, nb = plan.workspace(plan.workspace_size(CALL_MISFIT_GRAD_25D, nfreq * nk, nsrc, nrec))
    kyc = (ctypes.c_double * nk)(*ky.tolist())
    ckc = (ctypes.c_double * nk)(*ck.tolist())
    code = lib().helm_misfit_and_gradient_25d(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, kyc, ckc, nk,
                                              _ptr(src_idx), src_idx.numel(), _ptr(Q), nsrc, _ptr(wavelet),
                                              _ptr(rec_idx), nrec, _ptr(d_obs), _ptr(f), _ptr(g), ws, nb, rep,
                                              _stream(dev))
    _check(code, "helm_misfit_and_gradient_25d", allow_noconv=True)
    return f, g, reports_to_list(rep)


def wri_misfit_and_gradient(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, lam, cg_tol=1e-10,
                            cg_maxit=200, wavelet=None):
    """WRI (penalty) objective and gradient; the field of every pair comes from
    receiver-space conjugate gradients.  Returns (f [1], g [n_phys], reports)."""
    _dev(m_phys, torch.float64, "m_phys")
    _dev(src_idx, torch.int32, "src_idx")
    _dev(Q, torch.complex128, "Q")
    _dev(rec_idx, torch.int32, "rec_idx")
    _dev(d_obs, torch.complex128, "d_obs")
    if wavelet is not None:
        _dev(wavelet, torch.complex128, "wavelet")
    nfreq = len(np.atleast_1d(freqs_hz))
    _check_common(plan, m_phys, src_idx, Q, wavelet, nfreq)
    nsrc, nrec = Q.shape[1], rec_idx.numel()
    _need(tuple(d_obs.shape) == (nfreq, nsrc, nrec), "d_obs must be [nfreq, nsrc, nrec]")
    dev = m_phys.device
    f = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(plan.n_phys, dtype=torch.float64, device=dev)
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(CALL_WRI, nfreq, nsrc, nrec))
    code = lib().helm_wri_misfit_and_gradient(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(src_idx),
                                              src_idx.numel(), _ptr(Q), nsrc, _ptr(wavelet), _ptr(rec_idx), nrec,
                                              _ptr(d_obs), float(lam), float(cg_tol), int(cg_maxit), _ptr(f), _ptr(g),
                                              ws, nb, rep, _stream(dev))
    _check(code, "helm_wri_misfit_and_gradient", allow_noconv=True)
    return f, g, reports_to_list(rep)


def helm_misfit(plan: Plan, m_phys, freqs_hz, src_idx, Q, rec_idx, d_obs, wavelet=None, mask=None,
                keep_residuals=False, keep_fields=False, f_out=None, field_dtype=torch.complex128):
    """f only (one solve per pair); optionally the data residuals R [nfreq, nsrc, nrec]
    and forward fields U [nfreq, nsrc, n_comp] the gradient needs, stored as
    `field_dtype` (complex128, or complex64 at half the memory).
    Returns (f, R or None, U or None, reports)."""
    _need(field_dtype in (torch.complex128, torch.complex64), "field_dtype must be complex128 or complex64")
    _dev(m_phys, torch.float64, "m_phys")
    _dev(src_idx, torch.int32, "src_idx")
    _dev(Q, torch.complex128, "Q")
    _dev(rec_idx, torch.int32, "rec_idx")
    _dev(d_obs, torch.complex128, "d_obs")
    if wavelet is not None:
        _dev(wavelet, torch.complex128, "wavelet")
    if mask is not None:
        _dev(mask, torch.uint8, "mask")
    nfreq = len(np.atleast_1d(freqs_hz))
    _check_common(plan, m_phys, src_idx, Q, wavelet, nfreq)
    nsrc = Q.shape[1]
    nrec = rec_idx.numel()
    _need(tuple(d_obs.shape) == (nfreq, nsrc, nrec), "d_obs must be [nfreq, nsrc, nrec]")
    if mask is not None:
        _need(mask.numel() == nfreq * nsrc, "mask must be [nfreq, nsrc]")
    dev = m_phys.device
    f = torch.empty(1, dtype=torch.float64, device=dev) if f_out is None else f_out
    R = torch.empty((nfreq, nsrc, nrec), dtype=torch.complex128, device=dev) if keep_residuals else None
    U = torch.zeros((nfreq, nsrc, plan.n_comp), dtype=field_dtype, device=dev) if keep_fields else None
    u_type = FIELD_C64 if field_dtype == torch.complex64 else FIELD_C128
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(CALL_MISFIT, nfreq, nsrc, nrec))
    code = lib().helm_misfit(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(src_idx), src_idx.numel(),
                             _ptr(Q), nsrc, _ptr(wavelet), _ptr(rec_idx), nrec, _ptr(d_obs), _ptr(mask), _ptr(f),
                             _ptr(R), _ptr(U), u_type, ws, nb, rep, _stream(dev))
    _check(code, "helm_misfit", allow_noconv=True)
    return f, R, U, reports_to_list(rep)


def helm_gradient(plan: Plan, m_phys, freqs_hz, rec_idx, R, U, mask=None, g_out=None):
    """Adjoint-state gradient from stored residuals R and fields U (helm_misfit);
    U may be complex128 or complex64."""
    _dev(m_phys, torch.float64, "m_phys")
    _dev(rec_idx, torch.int32, "rec_idx")
    _dev(R, torch.complex128, "R")
    _need(isinstance(U, torch.Tensor) and U.dtype in (torch.complex128, torch.complex64),
          "U must be complex128 or complex64")
    _dev(U, U.dtype, "U")
    u_type = FIELD_C64 if U.dtype == torch.complex64 else FIELD_C128
    _check_common(plan, m_phys)
    nfreq, nsrc, nrec = R.shape
    _need(nfreq == len(np.atleast_1d(freqs_hz)) and nrec == rec_idx.numel(), "R must be [nfreq, nsrc, nrec]")
    _need(tuple(U.shape) == (nfreq, nsrc, plan.n_comp), "U must be [nfreq, nsrc, n_comp]")
    if mask is not None:
        _dev(mask, torch.uint8, "mask")
        _need(mask.numel() == nfreq * nsrc, "mask must be [nfreq, nsrc]")
    dev = m_phys.device
    g = torch.empty(plan.n_phys, dtype=torch.float64, device=dev) if g_out is None else g_out
    rep = _reports(nfreq * nsrc)
    ws, nb = plan.workspace(plan.workspace_size(CALL_GRADIENT, nfreq, nsrc, nrec))
    code = lib().helm_gradient(plan._h, _ptr(m_phys), _freqs(freqs_hz), nfreq, _ptr(rec_idx), nrec, _ptr(R), nsrc,
                               _ptr(U), u_type, _ptr(mask), _ptr(g), ws, nb, rep, _stream(dev))
    _check(code, "helm_gradient", allow_noconv=True)
    return g, reports_to_list(rep)


def misfit_and_gradient_batch(requests, nworkers: int = 4):
    """misfit_and_gradient for several models at once (helm_misfit_and_gradient_batch).

    `requests` is a list of dicts with keys plan, m_phys, freqs_hz, src_idx, Q,
    rec_idx, d_obs and optionally wavelet, mask.  Every request gets its own CUDA
    stream and workspace.  Returns a list of (f, g, reports)."""
    n = len(requests)
    _need(len({id(r["plan"]) for r in requests}) == n, "every request needs its own Plan (workspaces must not alias)")
    items = (HelmBatchItem * n)()
    keep, outs = [], []
    for i, r in enumerate(requests):
        plan = r["plan"]
        m, src, Q, rec, d = r["m_phys"], r["src_idx"], r["Q"], r["rec_idx"], r["d_obs"]
        wav, mask = r.get("wavelet"), r.get("mask")
        _dev(m, torch.float64, "m_phys")
        _dev(src, torch.int32, "src_idx")
        _dev(Q, torch.complex128, "Q")
        _dev(rec, torch.int32, "rec_idx")
        _dev(d, torch.complex128, "d_obs")
        nfreq = len(np.atleast_1d(r["freqs_hz"]))
        _check_common(plan, m, src, Q, wav, nfreq)
        nsrc, nrec = Q.shape[1], rec.numel()
        _need(tuple(d.shape) == (nfreq, nsrc, nrec), "d_obs must be [nfreq, nsrc, nrec]")
        f = torch.empty(1, dtype=torch.float64, device=m.device)
        g = torch.empty(plan.n_phys, dtype=torch.float64, device=m.device)
        rep = _reports(nfreq * nsrc)
        ws, nb = plan.workspace(plan.workspace_size(CALL_MISFIT_GRAD, nfreq, nsrc, nrec))
        stream = torch.cuda.Stream(device=m.device)
        fr = _freqs(r["freqs_hz"])
        it = items[i]
        it.plan = plan._h
        it.m_phys, it.freqs_hz, it.nfreq = m.data_ptr(), fr, nfreq
        it.src_idx, it.n_srcloc, it.Q, it.nsrc = src.data_ptr(), src.numel(), Q.data_ptr(), nsrc
        it.wavelet = wav.data_ptr() if wav is not None else None
        it.rec_idx, it.nrec, it.d_obs = rec.data_ptr(), nrec, d.data_ptr()
        it.mask = mask.data_ptr() if mask is not None else None
        it.f_out, it.g_out = f.data_ptr(), g.data_ptr()
        it.workspace, it.ws_bytes = ws.value, nb
        it.reports = rep
        it.stream = stream.cuda_stream
        keep.append((fr, stream))
        outs.append((f, g, rep))
    # the inputs were written on the caller's stream: make them visible to every item's stream
    torch.cuda.current_stream().synchronize()
    code = lib().helm_misfit_and_gradient_batch(items, n, int(nworkers))
    _check(code, "helm_misfit_and_gradient_batch", allow_noconv=True)
    return [(f, g, reports_to_list(rep)) for f, g, rep in outs]


def kernel_launch_count() -> int:
    return int(lib().helm_kernel_launch_count())


def profile_enable(on: bool = True):
    lib().helm_profile_enable(int(bool(on)))


def profile_read() -> dict:
    out = {}
    for i, name in enumerate(PROF_CLASSES):
        n, ms, by = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double()
        lib().helm_profile_read(i, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by))
        out[name] = dict(launches=int(n.value), ms=float(ms.value), bytes=float(by.value))
    return out
