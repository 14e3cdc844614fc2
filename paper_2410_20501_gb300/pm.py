"""Thin ctypes binding of libpmgb (include/pm_api.h) over torch device memory.

Argument marshalling only: every stage runs in the CUDA library.  torch
provides device memory (tensors, workspace) and the current CUDA stream.
If the library is missing this module raises instead of falling back.

Layouts: positions are uint32 fixed point stored in int32 tensors [3, np]
(same bits); velocities / accelerations float32 [3, np]; scalar grids float32
[n, n, n]; vector grids float32 [3, n, n, n].
"""
import ctypes
import math
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpmgb.so")

PM_WS_SORT, PM_WS_MG, PM_WS_FR, PM_WS_STEP, PM_WS_IDS, PM_WS_ADJ, PM_WS_FFT, PM_WS_LPT = 1, 2, 4, 8, 16, 32, 64, 128
PM_WS_REFINE = 256
PM_POISSON_MG, PM_POISSON_FFT7, PM_POISSON_FFT = 0, 1, 2
MG_GUESS_INPUT, MG_GUESS_JACOBI, MG_GUESS_SCALED = 0, 1, 2
PM_GRAVITY_NEWTON, PM_GRAVITY_FR, PM_GRAVITY_PARAM = 0, 1, 2
STATUS = {0: "PM_OK", 1: "PM_EINVAL", 2: "PM_ENOMEM", 3: "PM_ENOCONV", 4: "PM_ENAN", 5: "PM_ETIMEOUT",
          6: "PM_ECUDA", 7: "PM_EIO"}


class PMError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = f"{where}: {STATUS.get(code, code)}"
        if code == 6 and _lib is not None:
            msg += f" ({_lib.pm_last_cuda_error().decode()})"
        super().__init__(msg)


class mg_params(ctypes.Structure):
    _fields_ = [("npre", ctypes.c_int), ("npost", ctypes.c_int), ("omega", ctypes.c_float),
                ("coarsest", ctypes.c_int), ("coarse_max_sweeps", ctypes.c_int), ("coarse_drop", ctypes.c_float),
                ("max_cycles", ctypes.c_int), ("fixed_cycles", ctypes.c_int), ("tol", ctypes.c_double),
                ("stall", ctypes.c_double), ("first_guess", ctypes.c_int), ("guess_scale", ctypes.c_float),
                ("smoother", ctypes.c_int), ("coarse_omega", ctypes.c_float)]


class mg_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cycles", ctypes.c_int), ("norm_f", ctypes.c_double),
                ("res0", ctypes.c_double), ("res", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fr_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("Om", ctypes.c_double), ("OL", ctypes.c_double),
                ("fR0", ctypes.c_double), ("boxsize", ctypes.c_double), ("cycle", ctypes.c_int),
                ("npre", ctypes.c_int), ("npost", ctypes.c_int), ("coarsest", ctypes.c_int),
                ("coarse_max_sweeps", ctypes.c_int), ("coarse_drop", ctypes.c_float), ("cycles", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_cycles", ctypes.c_int), ("smoother", ctypes.c_int),
                ("nhs", ctypes.c_int)]


class pm_state(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("np", ctypes.c_int64), ("X", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("id", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("eps", ctypes.c_void_p),
                ("acc", ctypes.c_void_p), ("ws", ctypes.c_void_p), ("ws_bytes", ctypes.c_size_t),
                ("have_prev", ctypes.c_int)]


class pm_step_params(ctypes.Structure):
    _fields_ = [("a", ctypes.c_double), ("Om", ctypes.c_double), ("OL", ctypes.c_double),
                ("boxsize", ctypes.c_double), ("gravity", ctypes.c_int), ("fR0", ctypes.c_double),
                ("grad_order", ctypes.c_int), ("dt_kick", ctypes.c_double), ("dt_drift", ctypes.c_double),
                ("phi_rescale", ctypes.c_double), ("mg", mg_params), ("fr", fr_params), ("poisson", ctypes.c_int),
                ("mu0", ctypes.c_double), ("report_max", ctypes.c_int), ("serial", ctypes.c_int)]


class pm_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("mg", mg_stats), ("fr", mg_stats), ("max_acc", ctypes.c_double),
                ("max_vel", ctypes.c_double)]


class pm_batch_state(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("B", ctypes.c_int), ("np_box", ctypes.c_int64), ("X", ctypes.c_void_p),
                ("V", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t), ("have_prev", ctypes.c_int)]


class pm_batch_params(ctypes.Structure):
    _fields_ = [("grad_order", ctypes.c_int), ("src_scale", ctypes.c_void_p), ("dt_kick", ctypes.c_void_p),
                ("dt_drift", ctypes.c_void_p), ("phi_rescale", ctypes.c_void_p), ("mg", mg_params),
                ("cold_cycles", ctypes.c_int)]


_lib = None

_SIGS = {
    "pm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pm_last_cuda_error": (ctypes.c_char_p, []),
    "pm_version": (ctypes.c_char_p, []),
    "pm_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_size_t)]),
    "pm_sort": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pm_deposit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pm_deposit_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p]),
    "mg_default_params": (None, [ctypes.POINTER(mg_params)]),
    "mg_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(mg_params),
                                ctypes.POINTER(mg_stats), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "mg_solve_refine": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(mg_params), ctypes.POINTER(mg_stats), ctypes.c_void_p,
                                       ctypes.c_size_t, ctypes.c_void_p]),
    "fr_default_params": (None, [ctypes.POINTER(fr_params)]),
    "fr_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(fr_params),
                                ctypes.POINTER(mg_stats), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pm_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "pm_interp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                 ctypes.c_void_p]),
    "pm_step": (ctypes.c_int, [ctypes.POINTER(pm_state), ctypes.POINTER(pm_step_params), ctypes.POINTER(pm_stats),
                               ctypes.c_void_p]),
    "pm_step_host": (ctypes.c_int, [ctypes.POINTER(pm_state), ctypes.POINTER(pm_step_params),
                                    ctypes.POINTER(pm_stats), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "pm_deposit_adj": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "pm_interp_adj": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_size_t, ctypes.c_void_p]),
    "pm_gradient_adj": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p]),
    "mg_solve_adj": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(mg_params),
                                    ctypes.POINTER(mg_stats), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pm_poisson_fft": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pm_lpt2": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_size_t, ctypes.c_void_p]),
    "pm_batch_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "pm_step_batch": (ctypes.c_int, [ctypes.POINTER(pm_batch_state), ctypes.POINTER(pm_batch_params),
                                     ctypes.c_void_p]),
    "pm_deposit_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "mg_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(mg_params), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pm_fr_batch_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "fr_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(fr_params), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "pm_gradient_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p]),
    "pm_interp_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "pm_step_adj": (ctypes.c_int, [ctypes.POINTER(pm_state), ctypes.POINTER(pm_step_params), ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "pm_state_save": (ctypes.c_int, [ctypes.POINTER(pm_state), ctypes.c_char_p, ctypes.c_void_p]),
    "pm_state_load": (ctypes.c_int, [ctypes.POINTER(pm_state), ctypes.c_char_p, ctypes.c_void_p]),
    "pm_dt_supercomoving": (ctypes.c_double, [ctypes.c_double] * 4),
    "pm_growth_D": (ctypes.c_double, [ctypes.c_double] * 3),
    "pm_next_timestep": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double)]),
    "pm_max_speed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                    ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t,
                                    ctypes.c_void_p]),
    "pm_launch_count": (ctypes.c_uint64, []),
    "pm_timing_enable": (ctypes.c_int, [ctypes.c_int]),
    "pm_timing_collect": (ctypes.c_int, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_int]),
    "pm_autotune": (ctypes.c_int, [ctypes.c_int]),
    "pm_autotune_report": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
}


def lib():
    """Load libpmgb.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpmgb.so not built ({LIB_PATH}); run paper_2410_20501_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code, where):
    if code != 0:
        raise PMError(code, where)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t, dtype=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def positions_to_device(X, device="cuda"):
    """uint32 numpy [3, np] -> int32 CUDA tensor with the same bits."""
    return torch.from_numpy(np.ascontiguousarray(X, dtype=np.uint32).view(np.int32)).to(device)


def positions_to_host(t):
    return t.cpu().numpy().view(np.uint32)


def workspace_size(n, np_, flags):
    b = ctypes.c_size_t()
    _check(lib().pm_workspace_size(n, int(np_), flags, ctypes.byref(b)), "pm_workspace_size")
    return b.value


def workspace(n, np_, flags, device="cuda"):
    return torch.empty(workspace_size(n, np_, flags), dtype=torch.uint8, device=device)


def default_mg(**kw):
    p = mg_params()
    lib().mg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def default_fr(**kw):
    p = fr_params()
    lib().fr_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def sort(X, n, ws=None):
    """Stable cell sort: returns (perm int32 [np], cellstart int32 [n^3 + 1])."""
    np_ = X.shape[1]
    ws = ws if ws is not None else workspace(n, np_, PM_WS_SORT, X.device)
    perm = torch.empty(np_, dtype=torch.int32, device=X.device)
    cs = torch.empty(n ** 3 + 1, dtype=torch.int32, device=X.device)
    _check(lib().pm_sort(_p(X, torch.int32), np_, n, _p(perm), _p(cs), _p(ws), ws.numel(), _stream()), "pm_sort")
    return perm, cs


def deposit(X, n, ws=None):
    """TSC density rho~ [n, n, n] (mean 1)."""
    np_ = X.shape[1]
    ws = ws if ws is not None else workspace(n, np_, PM_WS_SORT, X.device)
    rho = torch.empty((n, n, n), dtype=torch.float32, device=X.device)
    _check(lib().pm_deposit(_p(X, torch.int32), np_, n, _p(rho), _p(ws), ws.numel(), _stream()), "pm_deposit")
    return rho


def mg_solve(f, phi=None, ws=None, **params):
    """Multigrid Poisson solve; returns (phi, stats dict)."""
    n = f.shape[0]
    prm = default_mg(**params)
    if phi is None:
        phi = torch.zeros_like(f)
        if "first_guess" not in params:
            prm.first_guess = MG_GUESS_JACOBI
    ws = ws if ws is not None else workspace(n, 0, PM_WS_MG, f.device)
    st = mg_stats()
    code = lib().mg_solve(_p(f, torch.float32), _p(phi, torch.float32), n, ctypes.byref(prm), ctypes.byref(st),
                          _p(ws), ws.numel(), _stream())
    if code not in (0, 3):
        _check(code, "mg_solve")
    return phi, st.as_dict()


def mg_solve_refine(f, phi=None, outer=3, ws=None, **params):
    """Poisson solve by iterative refinement: float64 phi (float32 multigrid
    corrections on float64 residuals); returns (phi, stats dict)."""
    n = f.shape[0]
    prm = default_mg(**params)
    phi = phi if phi is not None else torch.zeros(f.shape, dtype=torch.float64, device=f.device)
    ws = ws if ws is not None else workspace(n, 0, PM_WS_MG | PM_WS_REFINE, f.device)
    st = mg_stats()
    _check(lib().mg_solve_refine(_p(f, torch.float32), _p(phi, torch.float64), n, outer, ctypes.byref(prm),
                                 ctypes.byref(st), _p(ws), ws.numel(), _stream()), "mg_solve_refine")
    return phi, st.as_dict()


def fr_solve(rho, eps=None, ws=None, **params):
    """f(R) scalaron eps = u - 1; returns (eps, stats dict)."""
    n = rho.shape[0]
    prm = default_fr(**params)
    eps = eps if eps is not None else torch.zeros_like(rho)
    ws = ws if ws is not None else workspace(n, 0, PM_WS_FR, rho.device)
    st = mg_stats()
    code = lib().fr_solve(_p(rho, torch.float32), _p(eps, torch.float32), n, ctypes.byref(prm), ctypes.byref(st),
                          _p(ws), ws.numel(), _stream())
    if code not in (0, 3):
        _check(code, "fr_solve")
    return eps, st.as_dict()


def poisson_fft(rho, scale=1.0, kind=PM_POISSON_FFT7, ws=None):
    """phi = scale * G * (rho - <rho>) by the library's 3-D FFT (kind:
    PM_POISSON_FFT7 or PM_POISSON_FFT)."""
    n = rho.shape[0]
    ws = ws if ws is not None else workspace(n, 0, PM_WS_FFT, rho.device)
    phi = torch.empty_like(rho, dtype=torch.float32)
    _check(lib().pm_poisson_fft(_p(rho, torch.float32), _p(phi), n, kind, scale, _p(ws), ws.numel(), _stream()),
           "pm_poisson_fft")
    return phi


def lpt2(noise, amp, d1, e2, v1, v2, ws=None):
    """2LPT particles on the lattice from real white noise [n, n, n] and the
    amplitude grid [n, n, n//2+1] (device float32): returns (X int32 bits
    [3, n^3], V [3, n^3])."""
    n = noise.shape[0]
    ws = ws if ws is not None else workspace(n, 0, PM_WS_LPT, noise.device)
    X = torch.empty((3, n ** 3), dtype=torch.int32, device=noise.device)
    V = torch.empty((3, n ** 3), dtype=torch.float32, device=noise.device)
    _check(lib().pm_lpt2(_p(noise, torch.float32), _p(amp, torch.float32), n, d1, e2, v1, v2, _p(X), _p(V), _p(ws),
                         ws.numel(), _stream()), "pm_lpt2")
    return X, V


def gradient(phi, order=5):
    n = phi.shape[0]
    g = torch.empty((3, n, n, n), dtype=torch.float32, device=phi.device)
    _check(lib().pm_gradient(_p(phi, torch.float32), _p(g), n, order, _stream()), "pm_gradient")
    return g


def interp(g, X):
    n = g.shape[1]
    np_ = X.shape[1]
    acc = torch.empty((3, np_), dtype=torch.float32, device=X.device)
    _check(lib().pm_interp(_p(g, torch.float32), _p(X, torch.int32), np_, n, _p(acc), _stream()), "pm_interp")
    return acc


def deposit_adj(X, n, rho_bar):
    """Position cotangent [3, np] of pm_deposit given rho_bar [n, n, n]."""
    np_ = X.shape[1]
    out = torch.empty((3, np_), dtype=torch.float32, device=X.device)
    _check(lib().pm_deposit_adj(_p(X, torch.int32), np_, n, _p(rho_bar, torch.float32), _p(out), _stream()),
           "pm_deposit_adj")
    return out


def interp_adj(g, X, acc_bar, ws=None):
    """(g_bar [3, n, n, n], X cotangent [3, np]) of pm_interp given acc_bar."""
    n = g.shape[1]
    np_ = X.shape[1]
    ws = ws if ws is not None else workspace(n, np_, PM_WS_SORT | PM_WS_ADJ, X.device)
    g_bar = torch.empty_like(g)
    dX = torch.empty((3, np_), dtype=torch.float32, device=X.device)
    _check(lib().pm_interp_adj(_p(g, torch.float32), _p(X, torch.int32), np_, n, _p(acc_bar, torch.float32),
                               _p(g_bar), _p(dX), _p(ws), ws.numel(), _stream()), "pm_interp_adj")
    return g_bar, dX


def mg_solve_adj(phi_bar, ws=None, **params):
    """Cotangent of the source of a converged mg_solve given phi_bar: the
    same solve (the 7-point Laplacian is symmetric), from the Jacobi guess."""
    n = phi_bar.shape[0]
    prm = default_mg(**params)
    prm.first_guess = MG_GUESS_JACOBI
    f_bar = torch.zeros_like(phi_bar, dtype=torch.float32)
    ws = ws if ws is not None else workspace(n, 0, PM_WS_MG, phi_bar.device)
    st = mg_stats()
    code = lib().mg_solve_adj(_p(phi_bar, torch.float32), _p(f_bar), n, ctypes.byref(prm), ctypes.byref(st),
                              _p(ws), ws.numel(), _stream())
    if code not in (0, 3):
        _check(code, "mg_solve_adj")
    return f_bar


def gradient_adj(g_bar, order=5):
    n = g_bar.shape[1]
    phi_bar = torch.empty((n, n, n), dtype=torch.float32, device=g_bar.device)
    _check(lib().pm_gradient_adj(_p(g_bar, torch.float32), _p(phi_bar), n, order, _stream()), "pm_gradient_adj")
    return phi_bar


def next_timestep(a, Om, OL, n, max_acc, max_vel, courant=0.8, da_max=0.02, a_end=1.0):
    """pm_next_timestep: the §3.4 time step and the scale factor it reaches,
    (dt, a_next)."""
    dt, an = ctypes.c_double(), ctypes.c_double()
    _check(lib().pm_next_timestep(a, Om, OL, n, max_acc, max_vel, courant, da_max, a_end, ctypes.byref(dt),
                                  ctypes.byref(an)), "pm_next_timestep")
    return dt.value, an.value


def max_speed(V, n, ws, flags):
    """pm_max_speed: the largest |v| of V [3, np] (device), with a workspace
    sized by pm_workspace_size(n, np, flags)."""
    out = ctypes.c_double()
    _check(lib().pm_max_speed(_p(V, torch.float32), V.shape[1], n, flags, ctypes.byref(out), _p(ws), ws.numel(),
                              _stream()), "pm_max_speed")
    return out.value


def dt_supercomoving(Om, OL, a0, a1):
    return lib().pm_dt_supercomoving(Om, OL, a0, a1)


def growth_D(Om, OL, a):
    return lib().pm_growth_D(Om, OL, a)


def launch_count():
    return int(lib().pm_launch_count())


def timing_enable(on=True):
    _check(lib().pm_timing_enable(1 if on else 0), "pm_timing_enable")


TUNE_SITES = ("force_chunk", "mg_fused_chunk", "mg_smoother")


def autotune(mode):
    """pm_autotune: 0 fixed tilings, 1 tune batched launches (default), 2 forget and retune."""
    _check(lib().pm_autotune(int(mode)), "pm_autotune")


def autotune_report():
    """The tuned launch sites: [{site, n, B, chosen (None while undecided), samples}]."""
    cap = 64
    out = (ctypes.c_int * (5 * cap))()
    m = min(lib().pm_autotune_report(out, cap), cap)
    return [{"site": TUNE_SITES[out[5 * i]], "n": out[5 * i + 1], "B": out[5 * i + 2],
             "chosen": None if out[5 * i + 3] < 0 else out[5 * i + 3], "samples": out[5 * i + 4]}
            for i in range(m)]


def timing_collect():
    """{kernel class: (total ms, launches, algorithmic bytes)} since timing_enable()."""
    cap = 64
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = (ctypes.c_int64 * cap)()
    byt = (ctypes.c_double * cap)()
    k = lib().pm_timing_collect(names, ms, cnt, byt, cap)
    return {names[i].decode(): (ms[i], cnt[i], byt[i]) for i in range(k)}


class Simulation:
    """Device-resident particle state stepped by pm_step.

    X: uint32 numpy [3, np]; V: float32/float64 numpy [3, np].  Particles are
    kept in cell order (permuted every step); ``ids`` follows them if
    track_ids."""

    def __init__(self, X, V, n, Om, OL, boxsize, gravity="newton", fR0=-1e-5, grad_order=5, mg=None, fr=None,
                 track_ids=False, keep_acc=False, adjoint=False, poisson=0, mu0=0.0, device="cuda"):
        self.n = n
        self.np = X.shape[1]
        self.Om, self.OL, self.boxsize, self.fR0 = Om, OL, boxsize, fR0
        self.gravity = {"newton": PM_GRAVITY_NEWTON, "fr": PM_GRAVITY_FR, "mu": PM_GRAVITY_PARAM}[gravity]
        self.mu0 = mu0
        self.grad_order = grad_order
        self.X = positions_to_device(X, device)
        self.V = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float32)).to(device)
        self.ids = torch.arange(self.np, dtype=torch.int32, device=device) if track_ids else None
        self.phi = torch.zeros((n, n, n), dtype=torch.float32, device=device)
        self.eps = (torch.zeros((n, n, n), dtype=torch.float32, device=device)
                    if self.gravity == PM_GRAVITY_FR else None)
        self.acc = torch.empty((3, self.np), dtype=torch.float32, device=device) if keep_acc else None
        self.poisson = poisson
        self.serial = False   # True: scalaron solve on the caller's stream (per-kernel timing without overlap)
        flags = (PM_WS_STEP | (PM_WS_IDS if track_ids else 0) | (PM_WS_ADJ if adjoint else 0)
                 | (PM_WS_FFT if poisson else 0))
        self.ws = workspace(n, self.np, flags, device)
        self.ws_flags = flags
        self.mg = mg if mg is not None else default_mg()
        self.fr = fr if fr is not None else default_fr()
        self.state = pm_state(n=n, np=self.np, X=_p(self.X).value, V=_p(self.V).value,
                              id=_p(self.ids).value if track_ids else None, phi=_p(self.phi).value,
                              eps=_p(self.eps).value if self.eps is not None else None,
                              acc=_p(self.acc).value if keep_acc else None, ws=_p(self.ws).value,
                              ws_bytes=self.ws.numel(), have_prev=0)

    def params(self, a, dt_kick, dt_drift, phi_rescale=1.0, report_max=False):
        return pm_step_params(a=a, Om=self.Om, OL=self.OL, boxsize=self.boxsize, gravity=self.gravity,
                              fR0=self.fR0, grad_order=self.grad_order, dt_kick=dt_kick, dt_drift=dt_drift,
                              phi_rescale=phi_rescale, mg=self.mg, fr=self.fr, poisson=self.poisson, mu0=self.mu0,
                              report_max=1 if report_max else 0, serial=1 if self.serial else 0)

    def step(self, a, dt_kick, dt_drift, phi_rescale=1.0, report_max=False):
        st = pm_stats()
        prm = self.params(a, dt_kick, dt_drift, phi_rescale, report_max)
        code = lib().pm_step(ctypes.byref(self.state), ctypes.byref(prm), ctypes.byref(st), _stream())
        if code not in (0, 3):
            _check(code, "pm_step")
        out = {"status": st.status, "mg": st.mg.as_dict(), "fr": st.fr.as_dict()}
        if report_max:
            out["max_acc"], out["max_vel"] = st.max_acc, st.max_vel
        return out

    def run_adaptive(self, a_start, a_end, courant=0.8, da_max=0.02, max_steps=100000):
        """Kick-drift-kick from a_start to a_end with the time step of §3.4:
        courant * min(the step that raises a by da_max, sqrt(h / max|a|),
        h / max|v|), h = 1/n.  The fused kick of step i takes dt_i from the
        accelerations and velocities of step i - 1 (the first step from the
        initial velocities and the cosmological limit).  Returns the scale
        factors of the force evaluations (the last one is a_end, reached by a
        closing half kick)."""
        a = a_start
        max_vel = max_speed(self.V, self.n, self.ws, self.ws_flags)
        max_acc, dt_prev, out = 0.0, 0.0, [a_start]
        aD_prev = None
        for _ in range(max_steps):
            dt, a_next = next_timestep(a, self.Om, self.OL, self.n, max_acc, max_vel, courant, da_max, a_end)
            aD = a * growth_D(self.Om, self.OL, a)
            resc = aD / aD_prev if aD_prev is not None else 1.0
            st = self.step(a, 0.5 * (dt_prev + dt), dt, resc, report_max=True)
            max_acc, max_vel, dt_prev, aD_prev = st["max_acc"], st["max_vel"], dt, aD
            a = a_next
            out.append(a)
            if a >= a_end:
                break
        aD = a * growth_D(self.Om, self.OL, a)
        self.step(a, 0.5 * dt_prev, 0.0, aD / aD_prev)   # closing half kick at a_end
        return out

    def step_host(self, a, dt_kick, dt_drift, X_in, V_in, X_out, V_out, phi_rescale=1.0):
        """pm_step_host with pinned host tensors (int32 [3,np], float32 [3,np])."""
        st = pm_stats()
        prm = self.params(a, dt_kick, dt_drift, phi_rescale)
        code = lib().pm_step_host(ctypes.byref(self.state), ctypes.byref(prm), ctypes.byref(st),
                                  ctypes.c_void_p(X_in.data_ptr()), ctypes.c_void_p(V_in.data_ptr()),
                                  ctypes.c_void_p(X_out.data_ptr()), ctypes.c_void_p(V_out.data_ptr()), _stream())
        if code not in (0, 3):
            _check(code, "pm_step_host")
        return {"status": st.status, "mg": st.mg.as_dict(), "fr": st.fr.as_dict()}

    def run(self, a_steps, rescale_potential=True):
        """Kick-drift-kick through the scale factors a_steps (fused kicks):
        force at a_i, kick by (dt_{i-1} + dt_i)/2, drift by dt_i; a final
        half kick at a_N.  Returns per-step stats."""
        Om, OL = self.Om, self.OL
        dts = [dt_supercomoving(Om, OL, a_steps[i], a_steps[i + 1]) for i in range(len(a_steps) - 1)]
        D = [growth_D(Om, OL, a) for a in a_steps]
        out = []
        for i, a in enumerate(a_steps):
            prev = dts[i - 1] if i > 0 else 0.0
            cur = dts[i] if i < len(dts) else 0.0
            resc = (a * D[i]) / (a_steps[i - 1] * D[i - 1]) if (i > 0 and rescale_potential) else 1.0
            out.append(self.step(a, 0.5 * (prev + cur), cur, resc))
        return out

    def step_adjoint(self, a, dt_kick, dt_drift, X_bar_out, V_bar_out, phi=None):
        """Cotangents of this step's inputs (the current self.X, self.V, which
        are not modified) from the cotangents of its outputs (cell order of
        pm_step's output).  phi: the potential the forward step left in
        self.phi (None: recomputed, as a cold-started forward step would).
        Needs a workspace built with adjoint=True."""
        xb = torch.empty((3, self.np), dtype=torch.float32, device=self.X.device)
        vb = torch.empty_like(xb)
        prm = self.params(a, dt_kick, dt_drift)
        _check(lib().pm_step_adj(ctypes.byref(self.state), ctypes.byref(prm),
                                 None if phi is None else _p(phi, torch.float32), _p(X_bar_out, torch.float32),
                                 _p(V_bar_out, torch.float32), _p(xb), _p(vb), _stream()), "pm_step_adj")
        return xb, vb

    def save(self, path):
        """pm_state_save: checkpoint the particles, potentials and warm-start
        flag to a file."""
        _check(lib().pm_state_save(ctypes.byref(self.state), os.fsencode(path), _stream()), "pm_state_save")

    def load(self, path):
        """pm_state_load: resume from a checkpoint of a state of the same sizes."""
        _check(lib().pm_state_load(ctypes.byref(self.state), os.fsencode(path), _stream()), "pm_state_load")

    def positions(self):
        return positions_to_host(self.X)

    def velocities(self):
        return self.V.cpu().numpy()

    def particle_ids(self):
        return None if self.ids is None else self.ids.cpu().numpy()


def batch_workspace(n, B, np_box, device="cuda"):
    size = ctypes.c_size_t()
    _check(lib().pm_batch_workspace_size(n, B, np_box, ctypes.byref(size)), "pm_batch_workspace_size")
    return torch.empty(size.value, dtype=torch.uint8, device=device)


def deposit_batch(X, n, B, ws=None):
    """pm_deposit_batch: densities [B, n, n, n] of B boxes, X int32 bits [3, B * np_box]."""
    np_box = X.shape[1] // B
    ws = ws if ws is not None else batch_workspace(n, B, np_box, X.device)
    rho = torch.empty((B, n, n, n), dtype=torch.float32, device=X.device)
    _check(lib().pm_deposit_batch(_p(X, torch.int32), np_box, n, B, _p(rho), _p(ws), ws.numel(), _stream()),
           "pm_deposit_batch")
    return rho


def mg_solve_batch(f, phi=None, ws=None, **params):
    """mg_solve_batch: fixed V-cycles on B boxes, f [B, n, n, n]; returns phi."""
    B, n = f.shape[0], f.shape[1]
    prm = default_mg(**params)
    if phi is None:
        phi = torch.zeros_like(f)
        if "first_guess" not in params:
            prm.first_guess = MG_GUESS_JACOBI
    ws = ws if ws is not None else batch_workspace(n, B, 0, f.device)
    _check(lib().mg_solve_batch(_p(f, torch.float32), _p(phi, torch.float32), n, B, ctypes.byref(prm), _p(ws),
                                ws.numel(), _stream()), "mg_solve_batch")
    return phi


def fr_batch_workspace(n, B, device="cuda"):
    size = ctypes.c_size_t()
    _check(lib().pm_fr_batch_workspace_size(n, B, ctypes.byref(size)), "pm_fr_batch_workspace_size")
    return torch.empty(size.value, dtype=torch.uint8, device=device)


def fr_solve_batch(rho, eps=None, ws=None, **params):
    """fr_solve_batch: fixed FAS cycles on B boxes, rho [B, n, n, n] (shared parameters); returns eps."""
    B, n = rho.shape[0], rho.shape[1]
    prm = default_fr(**params)
    eps = eps if eps is not None else torch.zeros_like(rho)
    ws = ws if ws is not None else fr_batch_workspace(n, B, rho.device)
    _check(lib().fr_solve_batch(_p(rho, torch.float32), _p(eps, torch.float32), n, B, ctypes.byref(prm), _p(ws),
                                ws.numel(), _stream()), "fr_solve_batch")
    return eps


def gradient_batch(phi, order=5):
    B, n = phi.shape[0], phi.shape[1]
    g = torch.empty((B, 3, n, n, n), dtype=torch.float32, device=phi.device)
    _check(lib().pm_gradient_batch(_p(phi, torch.float32), _p(g), n, B, order, _stream()), "pm_gradient_batch")
    return g


def interp_batch(g, X):
    B, n = g.shape[0], g.shape[2]
    np_box = X.shape[1] // B
    acc = torch.empty((3, X.shape[1]), dtype=torch.float32, device=X.device)
    _check(lib().pm_interp_batch(_p(g, torch.float32), _p(X, torch.int32), np_box, n, B, _p(acc), _stream()),
           "pm_interp_batch")
    return acc


class Ensemble:
    """B independent boxes of n^3 cells stepped together by pm_step_batch.

    X: uint32 numpy [B, 3, np_box]; V: float [B, 3, np_box]; Om: [B] matter
    densities (flat: OL = 1 - Om).  Box b's particles occupy b*np_box ... in
    every plane of the device arrays and are kept in cell order within the box.
    step() is eager; capture() records one warm step in a CUDA graph that
    replay_step() then replays with the next coefficients."""

    def __init__(self, X, V, n, Om, boxsize, grad_order=5, mg=None, cold_cycles=8, device="cuda"):
        X = np.asarray(X, dtype=np.uint32)
        self.B, _, self.np_box = X.shape
        self.n, self.boxsize, self.grad_order, self.cold_cycles = n, boxsize, grad_order, cold_cycles
        self.Om = np.asarray(Om, dtype=np.float64).reshape(self.B)
        self.OL = 1.0 - self.Om
        npt = self.B * self.np_box
        self.X = torch.from_numpy(np.ascontiguousarray(X.transpose(1, 0, 2).reshape(3, npt)).view(np.int32)).to(device)
        self.V = torch.from_numpy(np.ascontiguousarray(
            np.asarray(V, dtype=np.float32).transpose(1, 0, 2).reshape(3, npt))).to(device)
        self.phi = torch.zeros((self.B, n, n, n), dtype=torch.float32, device=device)
        self.ws = batch_workspace(n, self.B, self.np_box, device)
        bpad = (self.B + 3) // 4 * 4                    # 16-byte aligned rows
        self.coef = torch.zeros((4, bpad), dtype=torch.float32, device=device)
        self.mg = mg if mg is not None else default_mg(fixed_cycles=2)
        self.state = pm_batch_state(n=n, B=self.B, np_box=self.np_box, X=_p(self.X).value, V=_p(self.V).value,
                                    phi=_p(self.phi).value, ws=_p(self.ws).value, ws_bytes=self.ws.numel(),
                                    have_prev=0)
        self.graph = None

    def coefficients(self, a_steps):
        """float32 [steps, 4, B]: per fused-kick step i and box b the source
        scale 3/2 a_i Om_b, the kick (dt_{i-1} + dt_i)/2, the drift dt_i and the
        warm-start factor a_i D_b(a_i) / (a_{i-1} D_b(a_{i-1})), dt in each
        box's supercomoving time."""
        S, B = len(a_steps) - 1, self.B
        out = np.zeros((S, 4, self.coef.shape[1]), dtype=np.float32)
        for b in range(B):
            Om, OL = float(self.Om[b]), float(self.OL[b])
            dts = [dt_supercomoving(Om, OL, a_steps[i], a_steps[i + 1]) for i in range(S)]
            aD = [a * growth_D(Om, OL, a) for a in a_steps]
            for i in range(S):
                out[i, 0, b] = 1.5 * a_steps[i] * Om
                out[i, 1, b] = 0.5 * ((dts[i - 1] if i > 0 else 0.0) + dts[i])
                out[i, 2, b] = dts[i]
                out[i, 3, b] = aD[i] / aD[i - 1] if i > 0 else 1.0
        return torch.from_numpy(out).to(self.coef.device)

    def _params(self):
        c = self.coef
        return pm_batch_params(grad_order=self.grad_order, src_scale=_p(c[0]).value, dt_kick=_p(c[1]).value,
                               dt_drift=_p(c[2]).value, phi_rescale=_p(c[3]).value, mg=self.mg,
                               cold_cycles=self.cold_cycles)

    def step(self, coef_row):
        """One eager step with the coefficients coef_row [4, B] (device)."""
        self.coef.copy_(coef_row)
        prm = self._params()
        _check(lib().pm_step_batch(ctypes.byref(self.state), ctypes.byref(prm), _stream()), "pm_step_batch")

    def capture(self):
        """Record one warm step (have_prev must be 1) in a CUDA graph."""
        if not self.state.have_prev:
            raise RuntimeError("capture a warm step: run one eager step first")
        prm = self._params()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            _check(lib().pm_step_batch(ctypes.byref(self.state), ctypes.byref(prm), _stream()), "pm_step_batch")
        self.graph = g

    def replay_step(self, coef_row):
        self.coef.copy_(coef_row)
        self.graph.replay()

    def positions(self):
        """uint32 [B, 3, np_box] (cell order within each box)."""
        X = positions_to_host(self.X).reshape(3, self.B, self.np_box)
        return np.ascontiguousarray(X.transpose(1, 0, 2))

    def velocities(self):
        V = self.V.cpu().numpy().reshape(3, self.B, self.np_box)
        return np.ascontiguousarray(V.transpose(1, 0, 2))

