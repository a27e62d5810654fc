"""ctypes front end of the FP64 CPU oracle (``pclb_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product package.  It shares no
code with the CUDA library.

Problems are described by any object with the attributes of
``paper_1302_7104_gb300.inputs.Workload`` (duck-typed; this package does not
import the product).  Arrays are float64: fields ``[n_theta][n_r]``,
distributions ``[Q][n_theta][n_r]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pclb_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libpclb_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_NONPHYS = 1
ORC_NONFINITE = 2
ORC_EINVAL = 4


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP contraction off, OpenMP on)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32),
        ("n_dirs", ctypes.c_int32), ("n_f", ctypes.c_int32),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
        ("speeds", ctypes.c_double * 5), ("B", ctypes.c_double * 5),
        ("tau", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc_kind", ctypes.c_int32 * 2),
        ("bc_values", ctypes.POINTER(ctypes.c_double) * 2),
        ("scheme", ctypes.c_int32), ("relaxation", ctypes.c_int32),
    ]


_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            L.orc_q.restype = ctypes.c_int
            L.orc_mwb_increment.restype = ctypes.c_double
            L.orc_mwb_increment.argtypes = [ctypes.c_double] * 6
            L.orc_scheme_increment.restype = ctypes.c_double
            L.orc_scheme_increment.argtypes = [ctypes.c_int] + [ctypes.c_double] * 6
            for name in ("orc_step", "orc_run", "orc_set_state", "orc_fields", "orc_diagnostics",
                         "orc_step_jvp", "orc_adjoint_step", "orc_set_state_jvp", "orc_fields_jvp",
                         "orc_step_nodes", "orc_adjoint_entries", "orc_noneq"):
                getattr(L, name).restype = ctypes.c_int
        return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Problem:
    """Holds the ctypes problem struct and keeps its BC arrays alive."""

    def __init__(self, w, tau=None, dt=None):
        self.w = w
        p = _Problem()
        p.n_r, p.n_theta = int(w.n_r), int(w.n_theta)
        p.n_dirs, p.n_f = int(w.n_dirs), int(w.n_f)
        p.r_in, p.r_out = float(w.r_in), float(w.r_out)
        p.speeds[:] = [float(x) for x in w.speeds]
        p.B[:] = [float(x) for x in w.B]
        p.tau = float(w.tau if tau is None else tau)
        p.dt = float(w.dt if dt is None else dt)
        self._keep = []
        for s in range(2):
            p.bc_kind[s] = int(w.bc_kind[s])
            v = w.bc_values[s]
            if v is not None:
                v = np.ascontiguousarray(v, dtype=np.float64)
                self._keep.append(v)
                p.bc_values[s] = _ptr(v)
            else:
                p.bc_values[s] = ctypes.cast(None, _dp)
        p.scheme = int(getattr(w, "scheme", 0))
        p.relaxation = int(getattr(w, "relaxation", 0))
        self.p = p
        self.Q = 1 + 4 * p.n_dirs
        self.shape = (self.Q, p.n_theta, p.n_r)

    @property
    def ref(self):
        return ctypes.byref(self.p)


def _check(st, what):
    if st & ORC_EINVAL:
        raise ValueError(f"oracle {what}: invalid problem")
    return st


def dvm(n_dirs=8, speeds=(0.0, 1.0, 2.92, 2.99, 4.49)):
    Q = 1 + 4 * n_dirs
    vx, vy = np.zeros(Q), np.zeros(Q)
    shell = np.zeros(Q, dtype=np.int32)
    sp = np.asarray(speeds, dtype=np.float64)
    lib().orc_dvm(ctypes.c_int(n_dirs), _ptr(sp), _ptr(vx), _ptr(vy),
                  shell.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return vx, vy, shell


def weights(E, n_dirs, speeds, B):
    F = np.zeros(5)
    lib().orc_weights(ctypes.c_int(n_dirs), _ptr(np.asarray(speeds, dtype=np.float64)),
                      _ptr(np.asarray(B, dtype=np.float64)), ctypes.c_double(E), _ptr(F))
    return F


def feq(rho, ux, uy, E, n_dirs, speeds, B):
    out = np.zeros(1 + 4 * n_dirs)
    lib().orc_feq(ctypes.c_int(n_dirs), _ptr(np.asarray(speeds, dtype=np.float64)),
                  _ptr(np.asarray(B, dtype=np.float64)), ctypes.c_double(rho), ctypes.c_double(ux),
                  ctypes.c_double(uy), ctypes.c_double(E), _ptr(out))
    return out


def moments(f, n_dirs, speeds):
    """(rho, u_x, u_y, E) of one node's distribution."""
    out = np.zeros(4)
    f = np.ascontiguousarray(f, dtype=np.float64)
    lib().orc_moments(ctypes.c_int(n_dirs), _ptr(np.asarray(speeds, dtype=np.float64)), _ptr(f), _ptr(out))
    return out


def mwb_increment(C, pm2, pm1, p0, pp1, pp2):
    return lib().orc_mwb_increment(C, pm2, pm1, p0, pp1, pp2)


SCHEME_MWB, SCHEME_WB, SCHEME_LW, SCHEME_UPWIND2 = 0, 1, 2, 3
RELAX_EXACT, RELAX_EULER = 0, 1


def scheme_increment(scheme, C, pm2, pm1, p0, pp1, pp2):
    """Increment M (psi^{n+1} = psi - M) of one convection scheme at one node."""
    return lib().orc_scheme_increment(int(scheme), C, pm2, pm1, p0, pp1, pp2)


def mwb_1d(psi, C):
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    out = np.zeros_like(psi)
    lib().orc_mwb_1d(ctypes.c_int(len(psi)), _ptr(psi), ctypes.c_double(C), _ptr(out))
    return out


def set_state(w, rho=None, u_r=None, u_theta=None, T=None, prob=None):
    prob = prob or Problem(w)
    fields = [np.ascontiguousarray(x if x is not None else d, dtype=np.float64)
              for x, d in zip((rho, u_r, u_theta, T), w.fields())]
    f = np.zeros(prob.shape)
    st = lib().orc_set_state(prob.ref, *[_ptr(x) for x in fields], _ptr(f))
    _check(st, "set_state")
    return f


def fields(w, f, prob=None):
    prob = prob or Problem(w)
    f = np.ascontiguousarray(f, dtype=np.float64)
    outs = [np.zeros((w.n_theta, w.n_r)) for _ in range(4)]
    _check(lib().orc_fields(prob.ref, _ptr(f), *[_ptr(o) for o in outs]), "fields")
    return tuple(outs)


def diagnostics(w, f, prob=None):
    prob = prob or Problem(w)
    out = np.zeros(6)
    f = np.ascontiguousarray(f, dtype=np.float64)
    _check(lib().orc_diagnostics(prob.ref, _ptr(f), _ptr(out)), "diagnostics")
    return out


def step(w, f, parallel=True, prob=None, return_status=False):
    prob = prob or Problem(w)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    st = _check(lib().orc_step(prob.ref, _ptr(f), _ptr(out), ctypes.c_int(int(parallel))), "step")
    return (out, st) if return_status else out


def run(w, f, n, parallel=True, prob=None, return_status=False):
    prob = prob or Problem(w)
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    st = _check(lib().orc_run(prob.ref, _ptr(f), ctypes.c_int(int(n)), ctypes.c_int(int(parallel))), "run")
    return (f, st) if return_status else f


def step_jvp(w, f, df, prob=None):
    prob = prob or Problem(w)
    f = np.ascontiguousarray(f, dtype=np.float64)
    df = np.ascontiguousarray(df, dtype=np.float64)
    out = np.empty_like(f)
    _check(lib().orc_step_jvp(prob.ref, _ptr(f), _ptr(df), _ptr(out)), "step_jvp")
    return out


def _ptr_array(arrs):
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
    arr = (_dp * len(keep))(*[_ptr(a) for a in keep])
    return arr, keep


def set_state_jvp(w, fields, dfields, prob=None):
    """d f^eq(fields) . dfields; fields, dfields: 4 arrays [n_theta][n_r]."""
    prob = prob or Problem(w)
    fa, k1 = _ptr_array(fields)
    da, k2 = _ptr_array(dfields)
    out = np.zeros(prob.shape)
    _check(lib().orc_set_state_jvp(prob.ref, fa, da, _ptr(out)), "set_state_jvp")
    return out


def fields_jvp(w, f, df, prob=None):
    """(d rho, d u_r, d u_theta, d T) = d fields(f) . df."""
    prob = prob or Problem(w)
    outs = [np.zeros((w.n_theta, w.n_r)) for _ in range(4)]
    oa, keep = _ptr_array(outs)
    f = np.ascontiguousarray(f, dtype=np.float64)
    df = np.ascontiguousarray(df, dtype=np.float64)
    _check(lib().orc_fields_jvp(prob.ref, _ptr(f), _ptr(df), oa), "fields_jvp")
    return tuple(keep)


def adjoint_step(w, f_n, lam_np1, prob=None):
    prob = prob or Problem(w)
    f_n = np.ascontiguousarray(f_n, dtype=np.float64)
    lam = np.ascontiguousarray(lam_np1, dtype=np.float64)
    out = np.empty_like(f_n)
    _check(lib().orc_adjoint_step(prob.ref, _ptr(f_n), _ptr(lam), _ptr(out)), "adjoint_step")
    return out


_ip = ctypes.POINTER(ctypes.c_int32)


def step_nodes(w, f, it, ir, prob=None):
    """f^{n+1} at the nodes (it[j], ir[j]) (0-based), shape [n, Q], from the
    whole f^n; the same operations as ``step``."""
    prob = prob or Problem(w)
    f = np.ascontiguousarray(f, dtype=np.float64)
    it = np.ascontiguousarray(it, dtype=np.int32)
    ir = np.ascontiguousarray(ir, dtype=np.int32)
    out = np.zeros((len(it), prob.Q))
    _check(lib().orc_step_nodes(prob.ref, _ptr(f), ctypes.c_int(len(it)), it.ctypes.data_as(_ip),
                                ir.ctypes.data_as(_ip), _ptr(out)), "step_nodes")
    return out


def adjoint_entries(w, f_n, lam_np1, q, it, ir, prob=None):
    """Entries lam^n[q[j], it[j], ir[j]] of the adjoint step (vector-Jacobian
    product), each by a node-local forward-mode sweep."""
    prob = prob or Problem(w)
    f_n = np.ascontiguousarray(f_n, dtype=np.float64)
    lam = np.ascontiguousarray(lam_np1, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.int32)
    it = np.ascontiguousarray(it, dtype=np.int32)
    ir = np.ascontiguousarray(ir, dtype=np.int32)
    out = np.zeros(len(q))
    _check(lib().orc_adjoint_entries(prob.ref, _ptr(f_n), _ptr(lam), ctypes.c_int(len(q)), q.ctypes.data_as(_ip),
                                     it.ctypes.data_as(_ip), ir.ctypes.data_as(_ip), _ptr(out)), "adjoint_entries")
    return out


NEQ_M, NEQ_DELTA, NEQ_MSTAR, NEQ_DSTAR = 1, 2, 4, 8
NEQ_COMPONENTS = ("2rr", "2rt", "2tt", "3rrr", "3rrt", "3rtt", "3ttt", "31r", "31t", "42rr", "42rt", "42tt")


def noneq(w, f, groups=15, prob=None):
    """Non-equilibrium manifestations of Sec. IV: for each selected group (bit
    0: M_m(f), 1: Delta_m, 2: M*_m(f), 3: Delta*_m) the 12 polar components
    of M_2, M_3, M_{3,1}, M_{4,2}; returns [n_groups, 12, n_theta, n_r]."""
    prob = prob or Problem(w)
    f = np.ascontiguousarray(f, dtype=np.float64)
    ng = bin(int(groups)).count("1")
    out = np.zeros((ng, 12, w.n_theta, w.n_r))
    _check(lib().orc_noneq(prob.ref, _ptr(f), ctypes.c_int(int(groups)), _ptr(out)), "noneq")
    return out
