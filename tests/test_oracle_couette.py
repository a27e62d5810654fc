"""The rotational-flow test of Sec. III A on the oracle: fluid between two
coaxial cylinders rotating with omega_1 = -0.1 (R1 = 1) and omega_2 = 0.1
(R2 = 2), computed on one sector (N_f = 1) with the rotated-label azimuthal
boundary, from rest to a steady state that the Navier-Stokes equations fix
as u_theta = A r + B / r (the no-slip solution, independent of viscosity).

The grid is a coarsened copy of the paper's 100 x 20 (50 x 10, dt = 2e-3,
the largest step the library's Courant check allows at this grid), run well
past the viscous spin-up time 1/(pi^2 nu) (nu = tau T).  The pins are the
shape of the profile (a least-squares fit of A r + B / r must leave only a
small residual) and its distance from the no-slip solution, which the
non-equilibrium boundary keeps within a few percent; with the equilibrium
ghost nodes the profile slips more at the walls (a Knudsen layer of the
order of the mean free path tau sqrt(T))."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I


def _steady(tau, steps, kind):
    w = I.taylor_couette(n_r=50, n_theta=10, tau=tau, dt=2e-3, bc_kind=kind)
    f = O.run(w, O.set_state(w), steps)
    rho, ur, ut, T = O.fields(w, f)
    r = I.radii(w.n_r, w.r_in, w.r_out)
    return r, ut.mean(axis=0), ut, ur, w


def _fit(r, u):
    M = np.stack([r, 1.0 / r], 1)
    c, *_ = np.linalg.lstsq(M, u, rcond=None)
    return c, np.max(np.abs(M @ c - u))


EXACT = np.array([(0.1 * 4 - (-0.1) * 1) / 3.0, 1 * 4 * (-0.1 - 0.1) / 3.0])   # A, B


def test_couette_profile_is_the_no_slip_solution_at_its_boundaries():
    r = np.linspace(1.0, 2.0, 11)
    u = I.couette_profile(r, -0.1, 0.1, 1.0, 2.0)
    assert u[0] == pytest.approx(-0.1) and u[-1] == pytest.approx(0.2)
    c, res = _fit(r, u)
    assert np.allclose(c, EXACT) and res < 1e-15


def test_steady_rotational_flow_with_non_equilibrium_boundary():
    r, prof, ut, ur, w = _steady(0.05, 20000, I.BC_WALL | I.BC_NEQ)
    exact = I.couette_profile(r, -0.1, 0.1, w.r_in, w.r_out)
    umax = np.max(np.abs(exact))
    c, res = _fit(r, prof)
    assert np.max(np.abs(prof - exact)) <= 0.05 * umax
    assert res <= 0.005 * umax                        # the profile has the form A r + B / r
    assert c[0] == pytest.approx(EXACT[0], rel=0.05)
    assert c[1] == pytest.approx(EXACT[1], rel=0.06)
    assert np.max(np.abs(ur)) <= 0.01 * umax          # no radial flow in the steady state


def test_equilibrium_ghosts_slip_more_than_non_equilibrium_ghosts():
    r, p_eq, *_ = _steady(0.01, 40000, I.BC_WALL)
    r, p_neq, _, _, w = _steady(0.01, 40000, I.BC_WALL | I.BC_NEQ)
    exact = I.couette_profile(r, -0.1, 0.1, w.r_in, w.r_out)
    umax = np.max(np.abs(exact))
    e_eq = np.max(np.abs(p_eq - exact)) / umax
    e_neq = np.max(np.abs(p_neq - exact)) / umax
    assert e_neq < e_eq <= 0.07
    assert _fit(r, p_eq)[1] <= 0.02 * umax


def test_non_equilibrium_flag_changes_nothing_at_equilibrium():
    # f = f^eq everywhere: the wall node's departure is zero (to rounding)
    for kind in (I.BC_EXTRAP, I.BC_WALL, I.BC_DIRICHLET):
        w = I.random_smooth(8, 6, seed=4, bc_kind=(kind, kind))
        if kind != I.BC_EXTRAP:
            w = I.taylor_couette(n_r=8, n_theta=6, bc_kind=kind)
        f = O.set_state(w)
        a = O.step(w, f)
        w.bc_kind = (kind | I.BC_NEQ, kind | I.BC_NEQ)
        b = O.step(w, f)
        assert np.max(np.abs(a - b)) <= 1e-15 * np.max(np.abs(a))


def test_non_equilibrium_flag_matters_away_from_equilibrium():
    w = I.random_smooth(8, 6, seed=5)
    f = O.set_state(w) * (1.0 + 0.05 * np.random.default_rng(5).normal(size=(33, 6, 8)))
    a = O.step(w, f)
    w.bc_kind = (I.BC_EXTRAP | I.BC_NEQ, I.BC_EXTRAP | I.BC_NEQ)
    b = O.step(w, f)
    diff = np.abs(a - b)
    assert np.max(diff[:, :, 2:-2]) == 0.0            # only the two nodes next to each wall read ghosts
    assert np.max(diff[:, :, :2]) > 1e-6 and np.max(diff[:, :, -2:]) > 1e-6
