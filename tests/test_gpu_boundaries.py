"""The boundary options beyond the basic ones on the GPU: the non-equilibrium
ghost nodes (PCLB_BC_NEQ, Sec. II C 1) against the oracle, in the step and
in its adjoint, and the
rotational-flow test of Sec. III A (rotating cylinders on one sector with the
rotated-label azimuthal boundary) against the oracle and against the steady
Navier-Stokes profile u_theta = A r + B / r."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NEQ = I.BC_NEQ
CASES = {
    "extrap_neq": lambda: I.random_smooth(37, 19, seed=1, bc_kind=(I.BC_EXTRAP | NEQ, I.BC_EXTRAP | NEQ)),
    "dirichlet_wall_neq": lambda: I.random_smooth(40, 24, seed=2, bc_kind=(I.BC_DIRICHLET | NEQ, I.BC_WALL | NEQ)),
    "couette_neq": lambda: I.taylor_couette(n_r=50, n_theta=10, tau=0.05, dt=2e-3, bc_kind=I.BC_WALL | NEQ),
    "mixed": lambda: I.random_smooth(33, 20, seed=6, bc_kind=(I.BC_WALL, I.BC_EXTRAP | NEQ)),
}


def _noisy(w, seed=11):
    f = O.set_state(w)
    return np.ascontiguousarray(f * (1.0 + 0.01 * np.random.default_rng(seed).normal(size=f.shape)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("name", list(CASES))
def test_neq_ghosts_one_step_match_oracle(name, prec, tol):
    w = CASES[name]()
    f0 = _noisy(w)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        f0 = f0.astype(np.float32).astype(np.float64)
    want = O.step(w, f0)
    with P.PCLB(w, precision=prec) as g:
        got = g.set_f(torch.as_tensor(f0, dtype=dtype, device="cuda")).step(1).get_f().double().cpu().numpy()
        assert g.status_flags() == 0
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= tol


@pytest.mark.parametrize("kind", [I.BC_WALL, I.BC_WALL | NEQ])
def test_couette_fp64_run_matches_oracle(kind):
    w = I.taylor_couette(n_r=50, n_theta=10, tau=0.05, dt=2e-3, bc_kind=kind)
    n = 2000
    want = O.fields(w, O.run(w, O.set_state(w), n))
    with P.PCLB(w, precision="fp64") as g:
        g.set_state().step(n)
        got = [x.cpu().numpy() for x in g.moments()]
        assert g.status_flags() == 0
    for a, b in zip(got, want):
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.max(np.abs(b)))


def test_couette_steady_state_on_gpu():
    w = I.taylor_couette(n_r=50, n_theta=10, tau=0.05, dt=2e-3, bc_kind=I.BC_WALL | NEQ)
    with P.PCLB(w, precision="fp32") as g:
        g.set_state().step(20000)
        rho, ur, ut, T = [x.double().cpu().numpy() for x in g.moments()]
        assert g.status_flags() == 0
    r = I.radii(w.n_r, w.r_in, w.r_out)
    exact = I.couette_profile(r, -0.1, 0.1, w.r_in, w.r_out)
    prof = ut.mean(axis=0)
    umax = np.max(np.abs(exact))
    M = np.stack([r, 1.0 / r], 1)
    c, *_ = np.linalg.lstsq(M, prof, rcond=None)
    assert np.max(np.abs(prof - exact)) <= 0.05 * umax
    assert np.max(np.abs(M @ c - prof)) <= 0.005 * umax
    assert np.max(np.abs(ur)) <= 0.01 * umax


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-4)])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_with_neq_boundaries_matches_oracle(name, prec, tol):
    """The adjoint step with non-equilibrium ghost nodes, every entry against
    the oracle's forward-mode derivative: the ghosts' cotangent reaches the
    wall node's f_q directly and, with the opposite sign, through its own
    equilibrium, besides the path through the extrapolated ghost state."""
    w = CASES[name]()
    f = _noisy(w)
    lam = np.random.default_rng(12).normal(size=f.shape)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        f = f.astype(np.float32).astype(np.float64)
        lam = lam.astype(np.float32).astype(np.float64)
    with P.PCLB(w, precision=prec) as g:
        got = g.adjoint_step(torch.as_tensor(f, dtype=dtype, device="cuda"),
                             torch.as_tensor(lam, dtype=dtype, device="cuda")).double().cpu().numpy()
        assert g.status_flags() == 0
    q, t, r = (a.ravel() for a in np.meshgrid(*(np.arange(n) for n in f.shape), indexing="ij"))
    want = O.adjoint_entries(w, f, lam, q, t, r).reshape(f.shape)
    err = np.abs(got - want) / np.max(np.abs(want))
    assert err.max() <= tol, (err.max(), np.unravel_index(np.argmax(err), err.shape))
