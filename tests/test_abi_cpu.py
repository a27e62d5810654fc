"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function the header declares, sizes its workspace and rejects invalid
arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "pclb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pclb_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    L = P.lib()
    declared = _declared()
    assert "pclb_step" in declared and "pclb_create" in declared
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(P.exported_symbols())
    assert L.pclb_version() == 1


def _grid_dvm(w):
    g = P.Grid(w.n_r, w.n_theta, w.r_in, w.r_out, w.n_f)
    d = P.Dvm(w.n_dirs, (ctypes.c_double * 5)(*w.speeds), (ctypes.c_double * 5)(*w.B))
    return g, d


def test_workspace_size_matches_layout():
    w = I.rot()
    g, d = _grid_dvm(w)
    n32, n64 = ctypes.c_size_t(), ctypes.c_size_t()
    assert P.lib().pclb_workspace_size(ctypes.byref(g), ctypes.byref(d), 0, ctypes.byref(n32)) == 0
    assert P.lib().pclb_workspace_size(ctypes.byref(g), ctypes.byref(d), 1, ctypes.byref(n64)) == 0
    pitch = 32 * ((w.n_r + 31) // 32)
    f_bytes = 33 * (w.n_theta + 4) * pitch * 4
    assert n32.value >= 2 * f_bytes and n64.value >= 4 * f_bytes
    assert n32.value % 256 == 0


def _create(w, dt=None, n_dirs=None, ws_bytes=1 << 40, workspace=256, prec=0):
    g, d = _grid_dvm(w)
    if n_dirs is not None:
        d.n_dirs = n_dirs
    bc = P.Bc()
    bc.kind[0], bc.kind[1] = 0, 0
    ctx = ctypes.c_void_p()
    code = P.lib().pclb_create(ctypes.byref(g), ctypes.byref(d), w.tau, w.dt if dt is None else dt, prec,
                               ctypes.byref(bc), ctypes.c_void_p(workspace), ws_bytes, None,
                               ctypes.byref(ctx))
    return code, P.lib().pclb_last_error(None).decode()


def test_create_rejects_invalid_arguments_without_a_device():
    w = I.uniform(8, 8)
    assert _create(w, dt=-1.0)[0] == 1                      # PCLB_EINVAL
    assert _create(w, dt=10.0)[0] == 6                      # PCLB_ECFL
    code, msg = _create(w, n_dirs=12)
    assert code == 8 and "n_dirs" in msg                    # PCLB_EUNSUPPORTED (8, 16, 24 only)
    assert _create(w, ws_bytes=1024)[0] == 2                # PCLB_ENOMEM
    assert _create(w, workspace=100)[0] == 1                # misaligned workspace
    bad = I.uniform(8, 8)
    bad.n_r = 2
    assert _create(bad)[0] == 1
    bad = I.uniform(8, 8)
    bad.r_in = 0.0
    assert _create(bad)[0] == 1


def test_courant_bound_of_the_workloads():
    # Every workload's dt passes the library's |C_r| + |C_theta| <= 1 check.
    for w in (I.rot(), I.shock(n_r=400), I.random_smooth(16, 16), I.kh(n_r=64, n_theta=64)):
        code, msg = _create(w, ws_bytes=1024)
        assert code == 2, msg   # gets past validation and Courant check, stops at the workspace size


def test_binding_refuses_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("CUDA present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        P.PCLB(I.uniform(8, 8))
