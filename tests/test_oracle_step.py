"""Pins of the oracle's full time step (combined scheme, Eq. 38, with the
boundary nodes of Sec. II C) against invariants, special cases, exact
solutions and grid convergence (no GPU)."""
import math
import sys
import os

import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I

sys.path.insert(0, os.path.dirname(__file__))
import riemann_exact  # noqa: E402


def _broadcast(fq, n_theta, n_r):
    return np.ascontiguousarray(np.broadcast_to(fq[:, None, None], (len(fq), n_theta, n_r)))


def test_uniform_state_stays_uniform():
    # Uniform rho, T and uniform *Cartesian* u: f^eq is the same at every node
    # when labels are Cartesian, every difference vanishes and only rounding
    # in the relaxation remains.
    w = I.uniform(9, 12)
    fq = O.feq(1.3, 0.31, -0.17, 0.9, 8, I.SPEEDS, I.TABLE1_B[8])
    f = _broadcast(fq, 12, 9)
    out = O.step(w, f)
    assert np.max(np.abs(out - f)) <= 1e-14 * np.max(np.abs(f))
    # interior nodes (stencils that reach no ghost) stay bitwise uniform
    assert np.all(out[:, :, 2:-2] == out[:, :1, 2:3])


def test_uniform_state_from_polar_fields():
    w = I.uniform(10, 16)
    f = O.set_state(w)
    out = O.run(w, f, 3)
    assert np.max(np.abs(out - f)) <= 1e-13 * np.max(np.abs(f))


def test_collision_conserves_mass_momentum_energy():
    # A spatially uniform non-equilibrium f has no differences to convect, so
    # one step is the relaxation of Eq. (19) alone; moments 1-3 of f^eq equal
    # those of f, hence rho, rho u and rho E are unchanged.
    rng = np.random.default_rng(2)
    w = I.uniform(6, 8, tau=3e-3)
    fq = O.feq(1.1, 0.2, 0.3, 0.8, 8, I.SPEEDS, I.TABLE1_B[8]) * (1 + 0.05 * rng.normal(size=33))
    f = _broadcast(fq, 8, 6)
    out = O.step(w, f)
    m0 = O.moments(fq, 8, I.SPEEDS)
    m1 = O.moments(out[:, 3, 2], 8, I.SPEEDS)
    assert m1 == pytest.approx(m0, rel=1e-13, abs=1e-14)
    feq = O.feq(*m0, 8, I.SPEEDS, I.TABLE1_B[8])
    decay = math.exp(-w.dt / w.tau)
    assert out[:, 3, 2] == pytest.approx(feq + (fq - feq) * decay, rel=1e-12, abs=1e-14)
    assert not np.allclose(out[:, 3, 2], fq, rtol=1e-6)  # relaxation did something


def test_relaxation_limits():
    rng = np.random.default_rng(4)
    fq = O.feq(0.9, -0.1, 0.25, 1.2, 8, I.SPEEDS, I.TABLE1_B[8]) * (1 + 0.05 * rng.normal(size=33))
    f = _broadcast(fq, 6, 6)
    feq = O.feq(*O.moments(fq, 8, I.SPEEDS), 8, I.SPEEDS, I.TABLE1_B[8])
    slow = O.step(I.uniform(6, 6, tau=1e30), f)      # tau -> infinity: nothing happens
    assert slow[:, 2, 2] == pytest.approx(fq, rel=1e-13, abs=1e-15)
    fast = O.step(I.uniform(6, 6, tau=1e-30), f)     # dt/tau -> infinity: f = f^eq
    assert fast[:, 2, 2] == pytest.approx(feq, rel=1e-13, abs=1e-15)


def _linear_fields(n_r, n_theta, r_in=1.0, r_out=2.0):
    R, TH = np.meshgrid(I.radii(n_r, r_in, r_out), I.angles(n_theta))
    lin = {"rho": lambda r: 1.0 + 0.1 * r, "u_r": lambda r: 0.1 + 0.02 * r,
           "u_t": lambda r: 0.3 - 0.05 * r, "T": lambda r: 0.8 + 0.05 * r}
    return R, lin


@pytest.mark.parametrize("kinds", [(I.BC_DIRICHLET, I.BC_DIRICHLET), (I.BC_WALL, I.BC_WALL),
                                   (I.BC_EXTRAP, I.BC_DIRICHLET)])
def test_radial_ghosts_extrapolate_linear_fields_exactly(kinds):
    # Fields linear in r: Eq. (39) extrapolation reproduces them at the ghost
    # radii, so extrapolated, prescribed and wall ghosts all give one result.
    n_r, n_t = 7, 8
    R, lin = _linear_fields(n_r, n_t)
    base = I.uniform(n_r, n_t)
    base.rho, base.u_r, base.u_theta, base.T = lin["rho"](R), lin["u_r"](R), lin["u_t"](R), lin["T"](R)
    gin, gout = I.ghost_radii(n_r, 1.0, 2.0)
    vals = []
    for gr in (gin, gout):
        v = np.zeros((2, 4, n_t))
        for layer, rg in enumerate(gr):
            v[layer] = np.array([lin["rho"](rg), lin["u_r"](rg), lin["u_t"](rg), lin["T"](rg)])[:, None]
        vals.append(v)
    f = O.set_state(base)
    ref = O.step(base, f)
    base.bc_kind, base.bc_values = kinds, tuple(vals)
    other = O.step(base, f)
    assert np.max(np.abs(other - ref)) <= 2e-13 * np.max(np.abs(ref))
    # and a wrong ghost value is seen by the rows next to the wall
    vals[0][0, 0, :] *= 1.01
    base.bc_kind, base.bc_values = (I.BC_DIRICHLET, I.BC_DIRICHLET), tuple(vals)
    wrong = O.step(base, f)
    assert np.max(np.abs(wrong[:, :, :2] - ref[:, :, :2])) > 1e-6
    assert np.max(np.abs(wrong[:, :, 2:] - ref[:, :, 2:])) <= 2e-13 * np.max(np.abs(ref))


def test_sector_with_label_rotation_matches_full_circle():
    # Eq. (40): a field with 8-fold symmetry computed on one sector (N_f = 1)
    # with rotated labels equals the first sector of the full-circle run.
    n_r, per_sector = 8, 3
    full = I.random_smooth(n_r, 8 * per_sector, seed=9)
    R, TH = np.meshgrid(I.radii(n_r, full.r_in, full.r_out), I.angles(8 * per_sector))
    x = (R - full.r_in) / (full.r_out - full.r_in)
    full.rho = 1.0 + 0.1 * np.cos(8 * TH) * (1 + x)
    full.T = 1.0 + 0.05 * np.sin(8 * TH + 0.3) * x
    full.u_r = 0.1 * np.sin(8 * TH) * x
    full.u_theta = 0.2 + 0.1 * np.cos(8 * TH) * x
    sector = I.random_smooth(n_r, per_sector, seed=9, n_f=1)
    sector.dt = full.dt
    for name in ("rho", "T", "u_r", "u_theta"):
        setattr(sector, name, np.ascontiguousarray(getattr(full, name)[:per_sector]))
    f_full = O.run(full, O.set_state(full), 4)
    f_sec = O.run(sector, O.set_state(sector), 4)
    assert np.max(np.abs(f_full[:, :per_sector] - f_sec)) <= 1e-13 * np.max(np.abs(f_sec))


def test_rigid_rotation_is_steady_to_first_order():
    # u_theta = 0.2 r with hydrostatic rho is an exact steady solution of the
    # Navier-Stokes limit (Eqs. 13-15); the drift at fixed time shrinks under
    # refinement (first-order scheme, appendix).
    drift = []
    for n_r, n_t in ((12, 24), (24, 48)):
        w = I.rot(n_r=n_r, n_theta=n_t)
        steps = int(round(0.36 / w.dt))
        f0 = O.set_state(w)
        f = O.run(w, f0, steps)
        rho, ur, ut, T = O.fields(w, f)
        drift.append(max(np.abs(ut - w.u_theta).max(), np.abs(rho - w.rho).max(), np.abs(ur).max()))
    assert drift[1] < 0.65 * drift[0], drift
    assert drift[1] < 2e-2


@pytest.mark.parametrize("pr", [10, 20])
def test_quasi_planar_shock_tube_matches_exact_riemann(pr):
    # A thin annulus at large radius is locally planar; the gamma = 2 Riemann
    # solution (Sec. III B setting) is the reference.  First-order smearing
    # only: L1 density error small, plateaus right.
    r_in, length, n_r = 1000.0, 1.0, 241
    w = I.shock(n_r=n_r, n_theta=4, r_in=r_in, r_out=r_in + length, r_split=r_in + 0.5,
                pressure_ratio=pr, tau=2e-5)
    t_end = 0.15
    steps = int(round(t_end / w.dt))
    f = O.run(w, O.set_state(w), steps)
    rho, ur, ut, T = O.fields(w, f)
    x = I.radii(n_r, r_in, r_in + length) - (r_in + 0.5)
    left, right = w.extra["left"], w.extra["right"]
    ex = riemann_exact.sample((left[0], 0.0, left[0] * left[2]), (right[0], 0.0, right[2]),
                              x / (steps * w.dt))
    l1 = np.mean(np.abs(rho[0] - ex[0]))
    assert l1 < 0.015, l1
    p_star, u_star = riemann_exact.star_state((1.0, 0.0, 1.0), (right[0], 0.0, right[2]))
    mid = np.abs(x - 0.5 * u_star * steps * w.dt) < 0.02   # just left of the contact
    assert np.all(np.abs(ur[0][mid] - u_star) < 0.01 * u_star)
    assert np.all(np.abs((rho * T)[0][mid] - p_star) < 0.01 * p_star)
    assert np.max(np.abs(ut)) < 1e-6          # no spurious swirl
    assert np.max(rho) <= 1.0 + 1e-3 and np.min(rho) >= right[0] - 1e-3   # no over/undershoot


def _front(x, a, lo, hi, region):
    """Positions in `region` where a crosses (lo + hi) / 2 (linear interpolation)."""
    idx = np.where(region)[0]
    s = a[idx] - 0.5 * (lo + hi)
    k = np.where(np.sign(s[:-1]) != np.sign(s[1:]))[0]
    return [x[idx[j]] - s[j] * (x[idx[j + 1]] - x[idx[j]]) / (s[j + 1] - s[j]) for j in k]


@pytest.mark.parametrize("pr", [10, 20])
def test_cylindrical_shock_tube_star_state_and_waves(pr):
    # The shock-tube workload itself (Sec. III B setting on r in [1, 3]):
    # 2000 x 16 nodes, 1000 steps (t = 0.056), jump at r = 2.  The geometry is
    # cylindrical, so the planar gamma = 2 Riemann solution holds only to
    # O(t c / r) ~ 4%: the star velocity to 1%, the star pressure to 4% (the
    # expanding shock weakens), the density in L1 to 1%.  Wave positions
    # within the scheme's smearing, sqrt(v_max dr t / 2) ~ 0.011: contact to
    # 0.005, shock (midpoint of the jump) to 0.02, rarefaction head to 0.015.
    w = I.shock(pressure_ratio=pr)
    steps = 1000
    t = steps * w.dt
    f = O.run(w, O.set_state(w), steps)
    rho, ur, ut, T = (a[0] for a in O.fields(w, f))   # one azimuthal row (the state is nearly axisymmetric)
    x = I.radii(w.n_r, w.r_in, w.r_out) - w.extra["r_split"]
    L, R = w.extra["left"], w.extra["right"]
    left, right = (L[0], 0.0, L[0] * L[2]), (R[0], 0.0, R[2])
    p_star, u_star = riemann_exact.star_state(left, right)
    ex = riemann_exact.sample(left, right, x / t)
    assert np.sum(np.abs(rho - ex[0])) / np.sum(np.abs(ex[0])) < 0.01
    star = (x > 0.2 * u_star * t) & (x < 0.8 * u_star * t)      # between rarefaction tail and contact
    assert np.all(np.abs(ur[star] - u_star) < 0.01 * u_star)
    assert np.all(np.abs((rho * T)[star] - p_star) < 0.04 * p_star)
    x_shock = x[np.where(np.abs(ex[0] - R[0]) > 1e-12)[0].max()]
    rho_s = ex[0][np.where(x < x_shock)[0].max()]              # density behind the shock
    shock = _front(x, rho, R[0], rho_s, x > u_star * t + 0.01)
    assert len(shock) == 1 and abs(shock[0] - x_shock) < 0.02, (shock, x_shock)
    rho_l = ex[0][np.argmin(np.abs(x - 0.5 * u_star * t))]     # left star density
    contact = _front(x, rho, rho_s, rho_l, (x > 0.005) & (x < x_shock - 0.01))
    assert len(contact) == 1 and abs(contact[0] - u_star * t) < 0.005, (contact, u_star * t)
    head = x[np.where(np.abs(ur) > 0.01 * u_star)[0].min()]
    assert abs(head + math.sqrt(2.0 * L[2]) * t) < 0.015, head


def test_grid_convergence_on_smooth_data():
    # Smooth radial acoustic pulse, three nested grids at fixed CFL: the
    # self-convergence order of rho is about one (first order, appendix).
    sols = []
    for n_r in (61, 121, 241):
        w = I.uniform(n_r, 4, rho=1.0, ux=0.0, uy=0.0, T=1.0, tau=2e-5, cfl=I.STABLE_CFL,
                      r_in=500.0, r_out=501.0)
        r = I.radii(n_r, 500.0, 501.0)
        bump = np.exp(-((r - 500.5) / 0.08) ** 2)
        w.rho = np.broadcast_to(1.0 + 0.02 * bump, (4, n_r)).copy()
        w.T = np.broadcast_to(1.0 + 0.01 * bump, (4, n_r)).copy()
        steps = int(round(0.1 / w.dt))
        w.dt = 0.1 / steps
        f = O.run(w, O.set_state(w), steps)
        sols.append(O.fields(w, f)[0][0])
    c, m, fne = sols
    e1 = np.abs(c - m[::2]).mean()
    e2 = np.abs(m[::2] - fne[::4]).mean()
    order = math.log2(e1 / e2)
    assert 0.8 < order < 2.5, (e1, e2, order)


def _entropy_blob_error(n_r, n_t, t_end=0.1, U=0.3, amp=0.2, sig=0.15, y0=1.5):
    """Mean |rho - exact| around a density blob carried by a uniform Cartesian
    flow U e_x through the annulus r in [1, 2] (uniform pressure: an exact
    Euler solution, rho(x - U t, y); heat conduction is O(tau) and negligible
    at tau = 2e-5).  At the top of the annulus the motion is azimuthal, so the
    blob's position tests C_theta = v_theta dt / (r dtheta) of Eq. (38)."""
    w = I.uniform(n_r, n_t, rho=1.0, ux=U, uy=0.0, T=1.0, tau=2e-5, cfl=I.STABLE_CFL, r_in=1.0, r_out=2.0)
    R, TH = np.meshgrid(I.radii(n_r, 1.0, 2.0), I.angles(n_t))
    X, Y = R * np.cos(TH), R * np.sin(TH)

    def rho_at(x):
        return 1.0 + amp * np.exp(-(x ** 2 + (Y - y0) ** 2) / sig ** 2)

    w.rho = rho_at(X)
    w.T = 1.0 / w.rho
    steps = int(math.ceil(t_end / w.dt))
    w.dt = t_end / steps
    rho = O.fields(w, O.run(w, O.set_state(w), steps))[0]
    near = X ** 2 + (Y - y0) ** 2 < (3 * sig) ** 2
    return np.abs(rho - rho_at(X - U * t_end))[near].mean()


def test_azimuthal_convection_converges_to_a_translated_blob():
    # Three nested grids (N_theta from 128 to 512; at r = 1.5, r dtheta is
    # 0.074 to 0.018 against a blob of width 0.15).  The error against the
    # exact translation falls at least first order (about second order is
    # seen: the limiter is inactive on smooth data) and ends below 0.25% of
    # the blob's amplitude.  Planted mistakes fail it: C_theta with R1 in
    # place of r stalls at order 0.2-0.6, a flipped v_theta does not converge.
    e = [_entropy_blob_error(n_r, n_t) for n_r, n_t in ((16, 128), (32, 256), (64, 512))]
    orders = [math.log2(e[0] / e[1]), math.log2(e[1] / e[2])]
    assert min(orders) >= 0.9, (e, orders)
    assert e[2] < 0.0025 * 0.2, e


def test_nonphysical_ghost_state_is_reported():
    # A steep density drop at the wall extrapolates to a negative ghost density.
    w = I.uniform(8, 4)
    R, _ = np.meshgrid(I.radii(8, w.r_in, w.r_out), I.angles(4))
    w.rho = np.where(R < 1.2, 1.0, 1.0) * np.where(np.isclose(R, w.r_in), 0.2, 1.0)
    f = O.set_state(w)
    _, status = O.step(w, f, return_status=True)
    assert status & O.ORC_NONPHYS


def test_invalid_problem_is_rejected():
    w = I.uniform(8, 4)
    w.tau = -1.0
    with pytest.raises(ValueError):
        O.step(w, np.zeros((33, 4, 8)))


def test_diagnostics_closed_form_for_uniform_state():
    # Sum over nodes of r dr dtheta: 2 pi dr (N R1 + dr N (N-1) / 2) for a full circle.
    n_r, n_t = 9, 12
    w = I.uniform(n_r, n_t, rho=1.3, ux=0.31, uy=-0.17, T=0.9)
    f = O.set_state(w)
    dr = (w.r_out - w.r_in) / (n_r - 1)
    area = 2 * math.pi * dr * (n_r * w.r_in + dr * n_r * (n_r - 1) / 2)
    m, jx, jy, e, rmin, tmin = O.diagnostics(w, f)
    assert m == pytest.approx(1.3 * area, rel=1e-13)
    assert jx == pytest.approx(1.3 * 0.31 * area, rel=1e-12)
    assert jy == pytest.approx(-1.3 * 0.17 * area, rel=1e-12)
    assert e == pytest.approx(1.3 * (0.9 + 0.5 * (0.31 ** 2 + 0.17 ** 2)) * area, rel=1e-12)
    assert rmin == pytest.approx(1.3, rel=1e-13) and tmin == pytest.approx(0.9, rel=1e-12)
