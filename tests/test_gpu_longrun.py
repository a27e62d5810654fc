"""The FP32 path over many steps at the workloads' full sizes, against the
FP64 GPU path (itself within 1e-12 per step of the oracle, see the parity
tests): the Kelvin-Helmholtz annulus 4096 x 4096 (smooth: relative L2 of rho,
u and T within 1e-5) and the Richtmyer-Meshkov annulus 1024 x 2048 (shocked:
relative L1 within 1e-4), each after hundreds of steps in the launch
configuration the benchmark times."""
import pytest

from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fields(w, prec, steps):
    with P.PCLB(w, precision=prec) as g:
        g.set_state().step(steps)
        assert g.status_flags() == 0
        rho, ur, ut, T = (x.double() for x in g.moments())
        g.sync()
        return rho, ur, ut, T


@pytest.mark.parametrize("name,steps,norm,tol", [("kh", 300, 2, 1e-5), ("rm", 600, 1, 1e-4)])
def test_fp32_long_run_tracks_fp64(name, steps, norm, tol):
    w = I.kh() if name == "kh" else I.rm()
    rho, ur, ut, T = _fields(w, "fp32", steps)
    rho_d, ur_d, ut_d, T_d = _fields(w, "fp64", steps)

    def rel(x, y):
        return (torch.linalg.vector_norm(x - y, ord=norm) / torch.linalg.vector_norm(y, ord=norm)).item()

    u, u_d = torch.stack([ur, ut]), torch.stack([ur_d, ut_d])
    errs = {"rho": rel(rho, rho_d), "u": rel(u.flatten(), u_d.flatten()), "T": rel(T, T_d)}
    print(name, steps, "steps, FP32 vs FP64:", errs)
    assert max(errs.values()) <= tol, errs
