"""Thin Python binding of the C ABI in ``include/pclb.h`` (ctypes).

Argument marshalling only: device memory and streams come from PyTorch, every
step of the computation runs in the library's CUDA kernels.  There is no CPU
fallback: without the compiled library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PCLB_FP32, PCLB_FP64 = 0, 1
STATUS = {0: "PCLB_OK", 1: "PCLB_EINVAL", 2: "PCLB_ENOMEM", 3: "PCLB_ECUDA", 4: "PCLB_ENONPHYS",
          5: "PCLB_ETIMEOUT", 6: "PCLB_ECFL", 7: "PCLB_ESTATE", 8: "PCLB_EUNSUPPORTED"}
FLAG_NONPHYS, FLAG_NONFINITE, FLAG_TIMEOUT = 1, 2, 4


# convection schemes and relaxations of pclb_set_scheme
SCHEME_MWB, SCHEME_WB, SCHEME_LW, SCHEME_UPWIND2 = 0, 1, 2, 3
RELAX_EXACT, RELAX_EULER = 0, 1

# groups of pclb_noneq and the order of its 12 components per group
NEQ_M, NEQ_DELTA, NEQ_MSTAR, NEQ_DSTAR = 1, 2, 4, 8
NEQ_COMPONENTS = ("2rr", "2rt", "2tt", "3rrr", "3rrt", "3rtt", "3ttt", "31r", "31t", "42rr", "42rt", "42tt")


class PCLBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32), ("r_in", ctypes.c_double),
                ("r_out", ctypes.c_double), ("n_f", ctypes.c_int32)]


class Dvm(ctypes.Structure):
    _fields_ = [("n_dirs", ctypes.c_int32), ("speeds", ctypes.c_double * 5), ("B", ctypes.c_double * 5)]


class Bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32 * 2), ("values", ctypes.POINTER(ctypes.c_double) * 2)]


_vp = ctypes.c_void_p
_SIGS = {
    "pclb_version": (ctypes.c_int32, []),
    "pclb_last_error": (ctypes.c_char_p, [_vp]),
    "pclb_workspace_size": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Dvm), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "pclb_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Dvm), ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, ctypes.POINTER(Bc), _vp, ctypes.c_size_t, _vp,
                                   ctypes.POINTER(_vp)]),
    "pclb_destroy": (ctypes.c_int, [_vp]),
    "pclb_set_stream": (ctypes.c_int, [_vp, _vp]),
    "pclb_set_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pclb_set_f": (ctypes.c_int, [_vp, _vp]),
    "pclb_get_f": (ctypes.c_int, [_vp, _vp]),
    "pclb_step": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "pclb_step_graph": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "pclb_step_states": (ctypes.c_int, [_vp, _vp, _vp]),
    "pclb_moments": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pclb_noneq": (ctypes.c_int, [_vp, ctypes.c_int32, _vp]),
    "pclb_set_scheme": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "pclb_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "pclb_diagnostics": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "pclb_status_flags": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32]),
    "pclb_sync": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "pclb_run_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp]),
    "pclb_state_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "pclb_save_state": (ctypes.c_int, [_vp, _vp]),
    "pclb_load_state": (ctypes.c_int, [_vp, _vp]),
    "pclb_lambda_set": (ctypes.c_int, [_vp, _vp]),
    "pclb_lambda_get": (ctypes.c_int, [_vp, _vp]),
    "pclb_adjoint_state": (ctypes.c_int, [_vp, _vp]),
    "pclb_adjoint_step": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "pclb_moments_vjp": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pclb_set_state_vjp": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pclb_diagnostics_noalloc": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Dvm), ctypes.c_int, _vp,
                                                ctypes.POINTER(ctypes.c_double), _vp]),
}


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libpclb.so (compiling it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and _build.stale():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype, fn.argtypes = res, args
            _lib = L
        return _lib


def _torch():
    import torch
    return torch


def _check(code: int, ctx=None):
    if code != 0:
        msg = lib().pclb_last_error(ctx).decode(errors="replace")
        raise PCLBError(code, msg)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


class PCLB:
    """One simulation context on one CUDA device.

    ``w`` is a workload (``paper_1302_7104_gb300.inputs.Workload`` or any
    object with its attributes); ``precision`` is "fp32" or "fp64".
    """

    def __init__(self, w, precision: str = "fp32", device=None, tau: Optional[float] = None,
                 dt: Optional[float] = None, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("PCLB needs a CUDA device; there is no CPU fallback")
        self.device = (torch.device(device) if device is not None
                       else torch.device("cuda", torch.cuda.current_device()))
        self.prec = {"fp32": PCLB_FP32, "fp64": PCLB_FP64}[precision]
        self.dtype = torch.float32 if self.prec == PCLB_FP32 else torch.float64
        self.w = w
        self.n_r, self.n_theta, self.q = int(w.n_r), int(w.n_theta), 1 + 4 * int(w.n_dirs)
        self._grid = Grid(self.n_r, self.n_theta, float(w.r_in), float(w.r_out), int(w.n_f))
        self._dvm = Dvm(int(w.n_dirs), (ctypes.c_double * 5)(*w.speeds), (ctypes.c_double * 5)(*w.B))
        self._keep = []
        bc = Bc()
        for s in range(2):
            bc.kind[s] = int(w.bc_kind[s])
            v = w.bc_values[s]
            if v is not None:
                arr = np.ascontiguousarray(v, dtype=np.float64)
                self._keep.append(arr)
                bc.values[s] = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._bc = bc
        L = lib()
        nbytes = ctypes.c_size_t()
        _check(L.pclb_workspace_size(ctypes.byref(self._grid), ctypes.byref(self._dvm), self.prec,
                                     ctypes.byref(nbytes)))
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) // 256 * 256
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            ctx = _vp()
            _check(L.pclb_create(ctypes.byref(self._grid), ctypes.byref(self._dvm),
                                 float(w.tau if tau is None else tau), float(w.dt if dt is None else dt),
                                 self.prec, ctypes.byref(bc), _vp(aligned), int(nbytes.value),
                                 _vp(self.stream.cuda_stream), ctypes.byref(ctx)))
        self.ctx = ctx
        scheme, relaxation = int(getattr(w, "scheme", 0)), int(getattr(w, "relaxation", 0))
        if scheme or relaxation:
            self.set_scheme(scheme, relaxation)

    def set_scheme(self, scheme: int = 0, relaxation: int = 0):
        """Convection scheme (SCHEME_*) and relaxation (RELAX_*) of later steps."""
        _check(lib().pclb_set_scheme(self.ctx, int(scheme), int(relaxation)), self.ctx)
        return self

    def set_wait_limit(self, limit_ns: int = 2_000_000_000):
        """Limit of a step kernel's wait for its own window copies (pclb_set_wait_limit)."""
        _check(lib().pclb_set_wait_limit(self.ctx, int(limit_ns)), self.ctx)
        return self

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            code = lib().pclb_destroy(self.ctx)
            self.ctx = None
            _check(code)

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                lib().pclb_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers -------------------------------------------------------------
    def _field(self, x):
        torch = _torch()
        t = torch.as_tensor(x, dtype=self.dtype, device=self.device).contiguous()
        if tuple(t.shape) != (self.n_theta, self.n_r):
            raise ValueError(f"field shape {tuple(t.shape)} != {(self.n_theta, self.n_r)}")
        return t

    def empty_field(self):
        return _torch().empty((self.n_theta, self.n_r), dtype=self.dtype, device=self.device)

    # -- calls ---------------------------------------------------------------
    def set_state(self, rho=None, u_r=None, u_theta=None, T=None):
        """f = f^eq of the fields (defaults: the workload's initial fields)."""
        w = self.w
        fs = [self._field(x if x is not None else d) for x, d in zip((rho, u_r, u_theta, T), w.fields())]
        _check(lib().pclb_set_state(self.ctx, *[_vp(_ptr(t)) for t in fs]), self.ctx)
        self._hold = fs   # keep inputs alive until the queued kernel has run
        return self

    def set_f(self, f):
        torch = _torch()
        t = torch.as_tensor(f, dtype=self.dtype, device=self.device).contiguous()
        if tuple(t.shape) != (self.q, self.n_theta, self.n_r):
            raise ValueError("f must be [Q][n_theta][n_r]")
        _check(lib().pclb_set_f(self.ctx, _vp(t.data_ptr())), self.ctx)
        self._hold = [t]
        return self

    def get_f(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.q, self.n_theta, self.n_r), dtype=self.dtype, device=self.device)
        _check(lib().pclb_get_f(self.ctx, _vp(out.data_ptr())), self.ctx)
        return out

    def step(self, n: int = 1):
        _check(lib().pclb_step(self.ctx, int(n)), self.ctx)
        return self

    def step_states(self, f_from, f_to):
        """One step from the saved state ``f_from`` into the buffer ``f_to``
        (both from ``new_state``/``save_state``); the context's state is left
        alone."""
        _check(lib().pclb_step_states(self.ctx, _vp(f_from.data_ptr()), _vp(f_to.data_ptr())), self.ctx)
        self._hold = (f_from, f_to)
        return self

    def step_graph(self, n: int = 1):
        """The same n steps as ``step``, launched as one CUDA graph (captured on
        first use for this n and state buffer, replayed afterwards)."""
        _check(lib().pclb_step_graph(self.ctx, int(n)), self.ctx)
        return self

    def moments(self, out: Optional[Sequence] = None):
        outs = list(out) if out is not None else [self.empty_field() for _ in range(4)]
        _check(lib().pclb_moments(self.ctx, *[_vp(_ptr(t)) for t in outs]), self.ctx)
        return tuple(outs)

    def noneq(self, groups: int = NEQ_M | NEQ_DELTA | NEQ_MSTAR | NEQ_DSTAR, out=None):
        """Non-equilibrium manifestations of the current state (Sec. IV):
        [n_groups, 12, n_theta, n_r] device tensor of the context's dtype,
        groups in bit order (NEQ_M, NEQ_DELTA, NEQ_MSTAR, NEQ_DSTAR), the 12
        polar components in the order of NEQ_COMPONENTS."""
        torch = _torch()
        ng = bin(int(groups) & 15).count("1")
        if out is None:
            out = torch.empty((ng, 12, self.n_theta, self.n_r), dtype=self.dtype, device=self.device)
        _check(lib().pclb_noneq(self.ctx, int(groups), _vp(out.data_ptr())), self.ctx)
        return out

    def diagnostics(self) -> np.ndarray:
        out = (ctypes.c_double * 8)()
        _check(lib().pclb_diagnostics(self.ctx, out), self.ctx)
        return np.array(out[:], dtype=np.float64)

    def status_flags(self, clear: bool = True, raise_on_error: bool = False) -> int:
        flags = ctypes.c_uint32()
        code = lib().pclb_status_flags(self.ctx, ctypes.byref(flags), int(clear))
        if code not in (0, 4, 5) or (raise_on_error and code != 0):
            _check(code, self.ctx)
        return int(flags.value)

    def sync(self, timeout_ms: int = 120000):
        _check(lib().pclb_sync(self.ctx, int(timeout_ms)), self.ctx)

    # -- reverse mode --------------------------------------------------------
    def state_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(lib().pclb_state_bytes(self.ctx, ctypes.byref(n)), self.ctx)
        return int(n.value)

    def new_state(self):
        """A device buffer for one stored state (uint8 tensor)."""
        return _torch().empty(self.state_bytes(), dtype=_torch().uint8, device=self.device)

    def save_state(self, buf=None):
        buf = self.new_state() if buf is None else buf
        _check(lib().pclb_save_state(self.ctx, _vp(buf.data_ptr())), self.ctx)
        return buf

    def load_state(self, buf):
        _check(lib().pclb_load_state(self.ctx, _vp(buf.data_ptr())), self.ctx)
        self._hold = [buf]
        return self

    def lambda_set(self, lam):
        torch = _torch()
        t = torch.as_tensor(lam, dtype=self.dtype, device=self.device).contiguous()
        if tuple(t.shape) != (self.q, self.n_theta, self.n_r):
            raise ValueError("lam must be [Q][n_theta][n_r]")
        _check(lib().pclb_lambda_set(self.ctx, _vp(t.data_ptr())), self.ctx)
        self._hold = [t]
        return self

    def lambda_get(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty((self.q, self.n_theta, self.n_r), dtype=self.dtype, device=self.device)
        _check(lib().pclb_lambda_get(self.ctx, _vp(out.data_ptr())), self.ctx)
        return out

    def adjoint_state(self, f_state=None):
        """lam <- J(f)^T lam for the state f saved in ``f_state`` (or the current one)."""
        _check(lib().pclb_adjoint_state(self.ctx, _vp(None if f_state is None else f_state.data_ptr())), self.ctx)
        return self

    def adjoint_step(self, f_n, lam_np1, out=None):
        torch = _torch()
        f = torch.as_tensor(f_n, dtype=self.dtype, device=self.device).contiguous()
        lam = torch.as_tensor(lam_np1, dtype=self.dtype, device=self.device).contiguous()
        if out is None:
            out = torch.empty_like(lam)
        _check(lib().pclb_adjoint_step(self.ctx, _vp(f.data_ptr()), _vp(lam.data_ptr()), _vp(out.data_ptr())),
               self.ctx)
        self._hold = [f, lam]
        return out

    def moments_vjp(self, g_rho=None, g_ur=None, g_ut=None, g_T=None):
        gs = [None if g is None else self._field(g) for g in (g_rho, g_ur, g_ut, g_T)]
        _check(lib().pclb_moments_vjp(self.ctx, *[_vp(_ptr(g)) for g in gs]), self.ctx)
        self._hold = gs
        return self

    def set_state_vjp(self, rho, u_r, u_theta, T):
        fs = [self._field(x) for x in (rho, u_r, u_theta, T)]
        outs = [self.empty_field() for _ in range(4)]
        _check(lib().pclb_set_state_vjp(self.ctx, *[_vp(_ptr(t)) for t in fs], *[_vp(_ptr(t)) for t in outs]),
               self.ctx)
        self._hold = fs
        return tuple(outs)

    def run_host(self, rho, u_r, u_theta, T, n: int, outs=None):
        """End-to-end call with host arrays (numpy or CPU tensors, ideally
        page-locked): upload, equilibrium, n steps, moments, download."""
        torch = _torch()
        ins = [torch.as_tensor(x, dtype=self.dtype).contiguous() for x in (rho, u_r, u_theta, T)]
        for t in ins:
            if t.device.type != "cpu" or tuple(t.shape) != (self.n_theta, self.n_r):
                raise ValueError("run_host takes host arrays of shape [n_theta][n_r]")
        if outs is None:
            outs = [torch.empty((self.n_theta, self.n_r), dtype=self.dtype) for _ in range(4)]
        _check(lib().pclb_run_host(self.ctx, *[_vp(t.data_ptr()) for t in ins], int(n),
                                   *[_vp(_ptr(t)) for t in outs]), self.ctx)
        return tuple(outs)


def diagnostics_noalloc(w, f, precision: str = "fp32", stream=None) -> np.ndarray:
    """Global integrals of the packed device distribution ``f`` ([Q][n_theta][n_r])
    through pclb_diagnostics_noalloc: no context and no device allocation, for
    callers that cannot allocate device memory.  Returns the 8 values of
    ``PCLB.diagnostics``."""
    torch = _torch()
    prec = {"fp32": PCLB_FP32, "fp64": PCLB_FP64}[precision]
    grid = Grid(int(w.n_r), int(w.n_theta), float(w.r_in), float(w.r_out), int(w.n_f))
    dvm = Dvm(int(w.n_dirs), (ctypes.c_double * 5)(*w.speeds), (ctypes.c_double * 5)(*w.B))
    if stream is None:
        stream = torch.cuda.current_stream(f.device)
    out = (ctypes.c_double * 8)()
    _check(lib().pclb_diagnostics_noalloc(ctypes.byref(grid), ctypes.byref(dvm), prec, _vp(f.data_ptr()),
                                          out, _vp(stream.cuda_stream)))
    return np.array(out[:], dtype=np.float64)


def exported_symbols():
    """Names of the functions the C ABI declares (for the loader test)."""
    return list(_SIGS)
