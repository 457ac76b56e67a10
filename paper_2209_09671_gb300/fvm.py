"""Thin ctypes binding of libfvm (include/fvm.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  PyTorch provides device memory (the workspace and the fields) and
the CUDA stream.  If the shared library is missing the import fails loudly;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfvm.so")

FVM_OK, FVM_EINVAL, FVM_ENOMEM, FVM_ECUDA, FVM_ENOCONV, FVM_EUNSTABLE, FVM_ETIMEOUT, \
    FVM_EUNSUPPORTED = range(8)
F64, MIXED = 0, 1


class fvm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("h", ctypes.c_double),
        ("bc", ctypes.c_int * 3),
        ("tbc", ctypes.c_int * 6),
        ("tbc_T0", ctypes.c_double * 6),
        ("tbc_dTamp", ctypes.c_double * 6),
        ("rho", ctypes.c_double * 2), ("mu", ctypes.c_double * 2),
        ("cp", ctypes.c_double * 2), ("lam", ctypes.c_double * 2),
        ("sigma0", ctypes.c_double), ("dsigma_dT", ctypes.c_double), ("T0", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("q_power", ctypes.c_double), ("q_radius", ctypes.c_double),
        ("q_x0", ctypes.c_double), ("q_y0", ctypes.c_double), ("q_speed", ctypes.c_double),
        ("cfl", ctypes.c_double), ("c_cap", ctypes.c_double), ("c_visc", ctypes.c_double),
        ("c_therm", ctypes.c_double), ("dt_max", ctypes.c_double),
        ("weno_eps", ctypes.c_double), ("weno_scale", ctypes.c_double * 3),
        ("smooth_passes", ctypes.c_int),
        ("mg_levels", ctypes.c_int), ("mg_pre", ctypes.c_int), ("mg_post", ctypes.c_int),
        ("mg_max_cycles", ctypes.c_int), ("mg_fixed_cycles", ctypes.c_int),
        ("mg_rtol", ctypes.c_double),
        ("coarse_rtol", ctypes.c_double), ("coarse_maxit", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("mx_inner_cycles", ctypes.c_int),
        ("adjoint", ctypes.c_int),
        ("concentration", ctypes.c_int),
        ("dsigma_dc", ctypes.c_double), ("c0", ctypes.c_double),
        ("diff_c", ctypes.c_double * 2),
        ("weno_scale_c", ctypes.c_double),
        ("alpha_scheme", ctypes.c_int),
        ("mg_coarse_sweeps", ctypes.c_int),
    ]


class fvm_state(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("T", ctypes.c_void_p), ("p", ctypes.c_void_p),
                ("c", ctypes.c_void_p)]


class fvm_step_info(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("dt_limiter", ctypes.c_int),
                ("vcycles", ctypes.c_int * 3), ("rel_residual", ctypes.c_double * 3),
                ("max_div_dt", ctypes.c_double), ("vol_sum", ctypes.c_double),
                ("mass_sum", ctypes.c_double), ("nan_flag", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"dt": self.dt, "dt_limiter": self.dt_limiter, "vcycles": list(self.vcycles),
                "rel_residual": list(self.rel_residual), "max_div_dt": self.max_div_dt,
                "vol_sum": self.vol_sum, "mass_sum": self.mass_sum, "nan_flag": self.nan_flag}


EXPORTS = ("fvm_workspace_size", "fvm_create", "fvm_destroy", "fvm_step", "fvm_poisson_solve",
           "fvm_step_adjoint", "fvm_status_string", "fvm_last_error", "fvm_version",
           "fvm_profile", "fvm_profile_read", "fvm_launch_count", "fvm_poisson_solve_noalloc",
           "fvm_stage_predict", "fvm_fma_peak", "fvm_sync")

KERNEL_CLASSES = ("smooth", "interface", "scalars", "momentum", "div_rhs", "beta", "gs_fine",
                  "gs_coarse", "restrict_fine", "restrict_coarse", "prolong_fine",
                  "prolong_coarse", "coarse_cg", "resnorm", "residual64", "add_correction",
                  "correct", "dt", "diagnostics", "misc", "adjoint", "coarse_tail")

_lib = None
FIELDS5 = ("u", "v", "w", "alpha", "T")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfvm.so (built by ``paper_2209_09671_gb300._build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfvm.so not found at {path}: build it with "
                           "paper_2209_09671_gb300._build.build(); there is no fallback")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.fvm_workspace_size.argtypes = [P(fvm_params), P(ctypes.c_size_t)]
    lib.fvm_create.argtypes = [P(fvm_params), ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                               P(ctypes.c_void_p)]
    lib.fvm_destroy.argtypes = [ctypes.c_void_p]
    lib.fvm_step.argtypes = [ctypes.c_void_p, P(fvm_state), ctypes.c_long, ctypes.c_double,
                             P(fvm_step_info)]
    lib.fvm_poisson_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, P(fvm_step_info)]
    lib.fvm_step_adjoint.argtypes = [ctypes.c_void_p, P(fvm_state), ctypes.c_long,
                                     ctypes.c_double, P(fvm_state), P(fvm_state),
                                     P(ctypes.c_double)]
    lib.fvm_status_string.argtypes = [ctypes.c_int]
    lib.fvm_status_string.restype = ctypes.c_char_p
    lib.fvm_last_error.argtypes = [ctypes.c_void_p]
    lib.fvm_last_error.restype = ctypes.c_char_p
    lib.fvm_version.restype = ctypes.c_char_p
    lib.fvm_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.fvm_launch_count.argtypes = [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_long)]
    lib.fvm_stage_predict.argtypes = [ctypes.c_void_p, P(fvm_state), ctypes.c_long,
                                      ctypes.c_double, P(ctypes.c_void_p), ctypes.c_void_p,
                                      ctypes.c_void_p]
    lib.fvm_poisson_solve_noalloc.argtypes = [P(fvm_params), ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, P(fvm_step_info)]
    lib.fvm_sync.argtypes = [ctypes.c_void_p]
    lib.fvm_fma_peak.argtypes = [ctypes.c_int, ctypes.c_void_p, P(ctypes.c_double),
                                 P(ctypes.c_double)]
    lib.fvm_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_int, P(ctypes.c_long),
                                     P(ctypes.c_double)]
    for name in ("fvm_workspace_size", "fvm_create", "fvm_destroy", "fvm_step",
                 "fvm_poisson_solve", "fvm_step_adjoint", "fvm_profile", "fvm_profile_read", "fvm_launch_count",
                 "fvm_poisson_solve_noalloc", "fvm_stage_predict", "fvm_fma_peak", "fvm_sync"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class FvmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def make_params(p) -> fvm_params:
    """Marshal a parameter object with the fields of ``cases.Params``."""
    c = fvm_params()
    c.nx, c.ny, c.nz, c.h = int(p.nx), int(p.ny), int(p.nz), float(p.h)
    c.bc[:] = [int(b) for b in p.bc]
    c.tbc[:] = [int(b) for b in p.tbc]
    c.tbc_T0[:] = [float(v) for v in p.tbc_T0]
    c.tbc_dTamp[:] = [float(v) for v in p.tbc_dTamp]
    c.rho[:], c.mu[:] = [float(v) for v in p.rho], [float(v) for v in p.mu]
    c.cp[:], c.lam[:] = [float(v) for v in p.cp], [float(v) for v in p.lam]
    c.sigma0, c.dsigma_dT, c.T0 = float(p.sigma0), float(p.dsigma_dT), float(p.T0)
    c.g[:] = [float(v) for v in p.g]
    c.q_power, c.q_radius = float(p.q_power), float(p.q_radius)
    c.q_x0, c.q_y0, c.q_speed = float(p.q_x0), float(p.q_y0), float(p.q_speed)
    c.cfl, c.c_cap, c.c_visc = float(p.cfl), float(p.c_cap), float(p.c_visc)
    c.c_therm, c.dt_max = float(p.c_therm), float(p.dt_max)
    c.weno_eps = float(p.weno_eps)
    c.weno_scale[:] = [float(v) for v in p.weno_scale]
    c.smooth_passes = int(p.smooth_passes)
    c.mg_levels, c.mg_pre, c.mg_post = int(p.mg_levels), int(p.mg_pre), int(p.mg_post)
    c.mg_max_cycles, c.mg_fixed_cycles = int(p.mg_max_cycles), int(p.mg_fixed_cycles)
    c.mg_rtol = float(p.mg_rtol)
    c.coarse_rtol, c.coarse_maxit = float(p.coarse_rtol), int(p.coarse_maxit)
    c.precision = int(p.precision)
    c.mx_inner_cycles = int(p.mx_inner_cycles)
    c.adjoint = int(getattr(p, "adjoint", 0))
    c.concentration = int(getattr(p, "concentration", 0))
    c.dsigma_dc = float(getattr(p, "dsigma_dc", 0.0))
    c.c0 = float(getattr(p, "c0", 0.0))
    c.diff_c[:] = [float(v) for v in getattr(p, "diff_c", (0.0, 0.0))]
    c.weno_scale_c = float(getattr(p, "weno_scale_c", 1.0))
    c.alpha_scheme = int(getattr(p, "alpha_scheme", 0))
    c.mg_coarse_sweeps = int(getattr(p, "mg_coarse_sweeps", 0))
    return c


def fvm_workspace_size(params) -> int:
    lib = load()
    n = ctypes.c_size_t(0)
    cp = params if isinstance(params, fvm_params) else make_params(params)
    st = lib.fvm_workspace_size(ctypes.byref(cp), ctypes.byref(n))
    if st != FVM_OK:
        raise FvmError(st, "fvm_workspace_size: invalid parameters")
    return n.value


class Solver:
    """A context bound to a torch-allocated workspace and a CUDA stream.

    ``fvm_step``, ``fvm_poisson_solve`` and ``fvm_step_adjoint`` forward to the
    C functions of the same names.  Fields are torch CUDA tensors: u, v, w,
    alpha, T in float64 (F64) or float32 (MIXED), p in float64.
    """

    def __init__(self, params, device="cuda", stream=None):
        import torch
        self.lib = load()
        self.params = params
        self.cparams = make_params(params)
        self.mixed = int(params.precision) == MIXED
        self.conc = int(getattr(params, "concentration", 0)) == 1
        self.rdtype = torch.float32 if self.mixed else torch.float64
        nbytes = fvm_workspace_size(self.cparams)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        ctx = ctypes.c_void_p()
        st = self.lib.fvm_create(ctypes.byref(self.cparams), ctypes.c_void_p(self.workspace.data_ptr()),
                                 ctypes.c_size_t(nbytes), ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(ctx))
        if st != FVM_OK:
            raise FvmError(st, "fvm_create failed")
        self.ctx = ctx

    def _check(self, st, what):
        if st != FVM_OK:
            msg = self.lib.fvm_last_error(self.ctx).decode()
            raise FvmError(st, f"{what}: {msg}")

    def _state(self, s, need_p=True) -> fvm_state:
        import torch
        st = fvm_state()
        for k in FIELDS5 + (("c",) if self.conc and "c" in s else ()):
            t = s[k]
            if not (t.is_cuda and t.dtype == self.rdtype and t.is_contiguous()):
                raise ValueError(f"field {k} must be a contiguous CUDA {self.rdtype} tensor")
            setattr(st, k, t.data_ptr())
        if not need_p:
            return st
        if not (s["p"].is_cuda and s["p"].dtype == torch.float64 and s["p"].is_contiguous()):
            raise ValueError("p must be a contiguous CUDA float64 tensor")
        st.p = s["p"].data_ptr()
        return st

    def fvm_step(self, state: dict, step_index: int = 0, dt: float = 0.0, info: bool = True,
                 raise_on_error: bool = True):
        st = self._state(state)
        inf = fvm_step_info() if info else None
        rc = self.lib.fvm_step(self.ctx, ctypes.byref(st), ctypes.c_long(step_index),
                               ctypes.c_double(dt), ctypes.byref(inf) if info else None)
        if raise_on_error:
            self._check(rc, "fvm_step")
        out = inf.as_dict() if info else {}
        out["status"] = rc
        return out

    def fvm_poisson_solve(self, alpha, rhs, p, raise_on_error: bool = True):
        inf = fvm_step_info()
        rc = self.lib.fvm_poisson_solve(self.ctx, ctypes.c_void_p(alpha.data_ptr()),
                                        ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                        ctypes.byref(inf))
        if raise_on_error:
            self._check(rc, "fvm_poisson_solve")
        out = inf.as_dict()
        out["status"] = rc
        return out

    def fvm_stage_predict(self, state: dict, step_index: int, dt: float) -> dict:
        """The first stage's predictor (no projection): returns u*, v*, w* and
        alpha + dt R_alpha, T + dt R_T as new tensors."""
        import torch
        st = self._state(state)
        out = {k: torch.empty_like(state[k]) for k in ("u", "v", "w", "alpha", "T")}
        us = (ctypes.c_void_p * 3)(out["u"].data_ptr(), out["v"].data_ptr(), out["w"].data_ptr())
        rc = self.lib.fvm_stage_predict(self.ctx, ctypes.byref(st), ctypes.c_long(step_index),
                                        ctypes.c_double(dt), us,
                                        ctypes.c_void_p(out["alpha"].data_ptr()),
                                        ctypes.c_void_p(out["T"].data_ptr()))
        self._check(rc, "fvm_stage_predict")
        return out

    def fvm_step_adjoint(self, state_n, step_index, dt, lam_np1, lam_n=None):
        """(lam_n, [dJ/d dsigma_dT, dJ/d q_power]) for one FP64 step at dt:
        lam_n = (dS_{n+1}/dS_n)^T lam_np1.  state_n holds u, v, w, alpha, T, p
        (read only); lam_np1 and lam_n hold u, v, w, alpha, T (float64 CUDA
        tensors); lam_n is allocated when None.  The context must have been
        created with ``adjoint = 1``."""
        import torch
        if lam_n is None:
            lam_n = {k: torch.empty_like(lam_np1[k]) for k in FIELDS5}
        dth = (ctypes.c_double * 2)(0.0, 0.0)
        rc = self.lib.fvm_step_adjoint(self.ctx, ctypes.byref(self._state(state_n)),
                                       ctypes.c_long(step_index), ctypes.c_double(dt),
                                       ctypes.byref(self._state(lam_np1, need_p=False)),
                                       ctypes.byref(self._state(lam_n, need_p=False)), dth)
        self._check(rc, "fvm_step_adjoint")
        return lam_n, [dth[0], dth[1]]

    def fvm_sync(self, raise_on_error: bool = True) -> int:
        """Wait for the solver's stream; the worst status of the device-side
        pressure solves since the last call (raises unless FVM_OK)."""
        rc = self.lib.fvm_sync(self.ctx)
        if raise_on_error:
            self._check(rc, "fvm_sync")
        return rc

    def fvm_profile(self, on: bool):
        self._check(self.lib.fvm_profile(self.ctx, 1 if on else 0), "fvm_profile")

    def fvm_profile_read(self) -> dict:
        """{class name: (launches, total ms)} since profiling was switched on."""
        out = {}
        for cls, name in enumerate(KERNEL_CLASSES):
            n = ctypes.c_long(0)
            ms = ctypes.c_double(0.0)
            self._check(self.lib.fvm_profile_read(self.ctx, cls, ctypes.byref(n), ctypes.byref(ms)),
                        "fvm_profile_read")
            out[name] = (n.value, ms.value)
        return out

    def fvm_launch_count(self, reset: bool = False) -> int:
        n = ctypes.c_long(0)
        self._check(self.lib.fvm_launch_count(self.ctx, 1 if reset else 0, ctypes.byref(n)),
                    "fvm_launch_count")
        return n.value

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fvm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fvm_poisson_solve_noalloc(params, alpha, rhs, p, stream=None) -> dict:
    """The allocation-free pressure solve (no context, no workspace): for
    callers that cannot allocate device memory.  alpha, rhs, p are CUDA
    tensors as for Solver.fvm_poisson_solve; the stream defaults to torch's
    current stream.  Returns the info dict with the status."""
    import torch
    lib = load()
    cp = params if isinstance(params, fvm_params) else make_params(params)
    n = int(cp.nx) * int(cp.ny) * int(cp.nz)
    adt = torch.float32 if int(cp.precision) == MIXED else torch.float64
    for name, t, dt in (("alpha", alpha, adt), ("rhs", rhs, torch.float64), ("p", p, torch.float64)):
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous() and t.device == p.device):
            raise ValueError(f"{name} must be a contiguous {dt} tensor on {p.device}")
        if t.numel() != n:
            raise ValueError(f"{name} must hold nx*ny*nz = {n} elements")
    with torch.cuda.device(p.device):
        if stream is None:
            stream = torch.cuda.current_stream(p.device)
        inf = fvm_step_info()
        rc = lib.fvm_poisson_solve_noalloc(ctypes.byref(cp), ctypes.c_void_p(alpha.data_ptr()),
                                           ctypes.c_void_p(rhs.data_ptr()),
                                           ctypes.c_void_p(p.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream), ctypes.byref(inf))
    out = inf.as_dict()
    out["status"] = rc
    return out


def fvm_fma_peak(precision: int, stream=None) -> dict:
    """Measured FMA throughput of the current device in double (F64) or
    float (MIXED): {"tflops": ..., "ms": ...}."""
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib.fvm_fma_peak(int(precision), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(tf),
                          ctypes.byref(ms))
    if rc != FVM_OK:
        raise FvmError(rc, "fvm_fma_peak failed")
    return {"tflops": tf.value, "ms": ms.value}


def to_device(state: dict, mixed: bool, device="cuda") -> dict:
    """Copy a host state (numpy float64 arrays) into CUDA tensors."""
    import torch
    rd = torch.float32 if mixed else torch.float64
    out = {}
    for k, v in state.items():
        t = torch.as_tensor(v)
        out[k] = t.to(device=device, dtype=torch.float64 if k == "p" else rd).contiguous()
    return out
