"""Seeded, synthetic inputs for the polar-coordinate FDLB step.

This module is shared by the CUDA path, its tests, the benchmark and the
oracle tests.  It holds *no* arithmetic of the method itself (no moments, no
equilibrium, no relaxation, no convection): it only builds the macroscopic
initial fields (rho, u_r, u_theta, T) on the paper's node positions, the
boundary values, and the problem constants (grid, velocity set, tau, dt).

Workloads (all synthetic PDE initial conditions; the paper uses no dataset):

* ``rot``    rigid rotation in an annulus (Sec. III A analogue)
* ``shock``  radial Riemann problem / shock tube (Sec. III B analogue)
* ``rm``     Richtmyer-Meshkov: perturbed material interface hit by a
             Mach-2 shock (Sec. III C analogue)
* ``rm_adj`` RM with a 16-mode interface built from seeded amplitudes
* ``kh``     Kelvin-Helmholtz shear layer (Sec. III D analogue)

Field arrays are float64 with shape ``[n_theta][n_r]`` (r fastest), the
layout the C ABI takes.

Node positions follow Sec. II C: r = R1 + (i_r - 1) dr with
dr = (R2 - R1) / (N_r - 1), i_r = 1..N_r (both walls are nodes), and
theta = i_theta * dtheta with dtheta = 2 pi N_f / (N_i N_theta),
i_theta = 1..N_theta.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

# Velocity set of Sec. II A: shell speeds v_0..v_4 and the octagon row of
# Table I.  B[n] is the coefficient of E^n in Eq. (11a); B[0] multiplies the
# shell weights in Eq. (11b).
SPEEDS = (0.0, 1.0, 2.92, 2.99, 4.49)
TABLE1_B = {
    8: (8.0, -0.25, 1.0, -6.0, 48.0),
    16: (16.0, -0.125, 0.5, -3.0, 24.0),
    24: (24.0, -1.0 / 12.0, 1.0 / 3.0, -2.0, 16.0),
}

# Courant number used by every workload (definition in dt_from_cfl).  When
# dt >> tau the additive combined scheme convects the non-equilibrium part of
# f undamped and is stable only up to about 1 - 1/sqrt(2) = 0.29.
STABLE_CFL = 0.25

BC_EXTRAP = 0     # rho, u, T linearly extrapolated (Eq. 39)
BC_WALL = 1       # rho, T extrapolated; u prescribed at the ghost nodes
BC_DIRICHLET = 2  # rho, u, T prescribed at the ghost nodes
BC_NEQ = 8        # flag added to a kind: ghosts also carry the wall node's f - f^eq

SCHEME_MWB, SCHEME_WB, SCHEME_LW, SCHEME_UPWIND2 = 0, 1, 2, 3
RELAX_EXACT, RELAX_EULER = 0, 1


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, velocity set, time step, BCs, fields."""

    name: str
    n_r: int
    n_theta: int
    r_in: float
    r_out: float
    tau: float
    dt: float
    steps: int
    rho: np.ndarray
    u_r: np.ndarray
    u_theta: np.ndarray
    T: np.ndarray
    n_dirs: int = 8
    n_f: int = 8
    speeds: tuple = SPEEDS
    B: tuple = TABLE1_B[8]
    bc_kind: tuple = (BC_EXTRAP, BC_EXTRAP)
    # per side: float64 [2 ghost layers][4 fields rho,u_r,u_theta,T][n_theta]
    # layer 0 is the ghost next to the wall, layer 1 the outer one.
    bc_values: tuple = (None, None)
    smooth: bool = True
    extra: dict = dataclasses.field(default_factory=dict)
    scheme: int = 0       # convection: SCHEME_MWB, _WB, _LW, _UPWIND2
    relaxation: int = 0   # RELAX_EXACT (Eq. 19) or RELAX_EULER

    @property
    def q(self) -> int:
        return 1 + 4 * self.n_dirs

    @property
    def cells(self) -> int:
        return self.n_r * self.n_theta

    def fields(self):
        return self.rho, self.u_r, self.u_theta, self.T


def radii(n_r: int, r_in: float, r_out: float) -> np.ndarray:
    """Node radii, i_r = 1..N_r (both walls included)."""
    dr = (r_out - r_in) / (n_r - 1)
    return r_in + np.arange(n_r, dtype=np.float64) * dr


def angles(n_theta: int, n_dirs: int = 8, n_f: int = 8) -> np.ndarray:
    """Node angles theta = i_theta * dtheta, i_theta = 1..N_theta."""
    dth = 2.0 * math.pi * n_f / (n_dirs * n_theta)
    return np.arange(1, n_theta + 1, dtype=np.float64) * dth


def ghost_radii(n_r: int, r_in: float, r_out: float):
    """Radii of the ghost layers (adjacent, outer) on the inner and outer side."""
    dr = (r_out - r_in) / (n_r - 1)
    return (r_in - dr, r_in - 2 * dr), (r_out + dr, r_out + 2 * dr)


def dt_from_cfl(cfl: float, n_r: int, n_theta: int, r_in: float, r_out: float,
                n_dirs: int = 8, n_f: int = 8, v_max: float = SPEEDS[-1]) -> float:
    """Time step for a Courant number of the *combined* (unsplit, additive)
    scheme: CFL = v_max dt (1/dr + 1/(R1 dtheta)).

    The paper gives dt directly.  The sum over both directions is used because
    the radial and azimuthal increments are added to the same node: the update
    stays a convex combination only while the two directional Courant numbers
    together stay below about one, and a per-direction definition
    (dt = CFL min(dr, R1 dtheta) / v_max) goes unstable at CFL >= 0.4 on the
    rotation workload.  With dt >> tau the relaxation removes the whole
    non-equilibrium part each step while the MWB increments of that part are
    added back undamped; the grid-scale mode then grows unless the summed
    Courant number stays below about 0.29, so all workloads use STABLE_CFL.
    """
    dr = (r_out - r_in) / (n_r - 1)
    dth = 2.0 * math.pi * n_f / (n_dirs * n_theta)
    return cfl / (v_max * (1.0 / dr + 1.0 / (r_in * dth)))


# --------------------------------------------------------------------------
# Shock relations (Eq. 45) for gamma = 2, E = T, P = rho T.  Used to build
# initial states only.
# --------------------------------------------------------------------------
GAMMA = 2.0


def hugoniot_from_speed(rho0: float, u0: float, p0: float, D: float):
    """Post-shock (rho, u, P) behind a shock of speed D into (rho0, u0, p0).

    Solves Eq. (45) with E = P / ((gamma - 1) rho): mass, momentum and the
    Hugoniot energy relation.  Closed form of the density ratio for an ideal
    gas; returns (rho_H, u_H, p_H).
    """
    g = GAMMA
    w = D - u0                      # shock speed relative to the pre-shock gas
    c0 = math.sqrt(g * p0 / rho0)
    m2 = (w / c0) ** 2
    ratio = (g + 1.0) * m2 / ((g - 1.0) * m2 + 2.0)
    rho_h = rho0 * ratio
    u_h = D - rho0 * w / rho_h      # rho_H (u_H - D) = rho0 (u0 - D)
    p_h = p0 + rho0 * w * (u_h - u0)
    return rho_h, u_h, p_h


def hugoniot_from_mach(rho0: float, u0: float, p0: float, mach: float, direction: float = 1.0):
    """Post-shock state and shock speed for a shock of Mach number ``mach``
    moving in ``direction`` (+1 outward, -1 inward) into a gas at rest-frame
    velocity u0.  Returns (rho_H, u_H, p_H, D)."""
    c0 = math.sqrt(GAMMA * p0 / rho0)
    D = u0 + direction * mach * c0
    rho_h, u_h, p_h = hugoniot_from_speed(rho0, u0, p0, D)
    return rho_h, u_h, p_h, D


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------
def _empty_bc():
    return (None, None)


def _mesh(n_r, n_theta, r_in, r_out, n_dirs=8, n_f=8):
    r = radii(n_r, r_in, r_out)
    th = angles(n_theta, n_dirs, n_f)
    R, TH = np.meshgrid(r, th)          # shape [n_theta][n_r]
    return R, TH


def rot(n_r: int = 32, n_theta: int = 64, steps: int = 200, cfl: float = STABLE_CFL,
        tau: float = 1e-4, omega: float = 0.2, r_in: float = 0.5, r_out: float = 1.5) -> Workload:
    """Rigid rotation u_theta = omega r, u_r = 0, T = 1 and
    rho = exp(omega^2 r^2 / 2) in hydrostatic balance (dP/dr = rho u^2 / r).
    Both walls are Dirichlet with the same state at the ghost radii."""
    R, _ = _mesh(n_r, n_theta, r_in, r_out)
    a = 0.5 * omega * omega
    rho = np.exp(a * R * R)
    u_r = np.zeros_like(R)
    u_th = omega * R
    T = np.ones_like(R)
    gin, gout = ghost_radii(n_r, r_in, r_out)
    vals = []
    for gr in (gin, gout):
        v = np.zeros((2, 4, n_theta))
        for layer, rg in enumerate(gr):
            v[layer, 0, :] = math.exp(a * rg * rg)
            v[layer, 1, :] = 0.0
            v[layer, 2, :] = omega * rg
            v[layer, 3, :] = 1.0
        vals.append(v)
    dt = dt_from_cfl(cfl, n_r, n_theta, r_in, r_out)
    return Workload("rot", n_r, n_theta, r_in, r_out, tau, dt, steps, rho, u_r, u_th, T,
                    bc_kind=(BC_DIRICHLET, BC_DIRICHLET), bc_values=tuple(vals))


def taylor_couette(n_r: int = 100, n_theta: int = 20, steps: int = 20000, tau: float = 0.2, dt: float = 1e-3,
                   omega_in: float = -0.1, omega_out: float = 0.1, r_in: float = 1.0, r_out: float = 2.0,
                   n_f: int = 1, bc_kind: int = BC_WALL) -> Workload:
    """Fluid between two coaxial cylinders rotating with angular velocities
    omega_in (r = R1) and omega_out (r = R2), Sec. III A: at rest in
    equilibrium at t = 0 with rho = 1, T = 1, on one sector (N_f = 1 of the
    N_i = 8 parts) with the rotated-label azimuthal boundary of Eq. (40).  Both
    radial boundaries are of kind ``bc_kind`` (WALL by default: rho and T
    extrapolated, u prescribed at the ghost nodes) with the ghost nodes moving
    with the cylinder, u_theta = omega r_ghost, u_r = 0.  The paper's run:
    N_r x N_theta = 100 x 20, dt = 1e-3, tau in {0.2, 0.1, 0.05, 0.01}; the
    steady state approaches u_theta = A r + B / r (``couette_profile``)."""
    R, _ = _mesh(n_r, n_theta, r_in, r_out, 8, n_f)
    rho = np.ones_like(R)
    zero = np.zeros_like(R)
    gin, gout = ghost_radii(n_r, r_in, r_out)
    vals = []
    for gr, om in ((gin, omega_in), (gout, omega_out)):
        v = np.zeros((2, 4, n_theta))
        for layer, rg in enumerate(gr):
            v[layer, 0, :] = 1.0
            v[layer, 2, :] = om * rg
            v[layer, 3, :] = 1.0
        vals.append(v)
    w = Workload("taylor_couette", n_r, n_theta, r_in, r_out, tau, dt, steps, rho, zero, zero.copy(),
                 np.ones_like(R), n_f=n_f, bc_kind=(bc_kind, bc_kind), bc_values=tuple(vals))
    w.extra = {"omega_in": omega_in, "omega_out": omega_out}
    return w


def couette_profile(r, omega_in: float, omega_out: float, r_in: float, r_out: float):
    """Steady azimuthal velocity between rotating cylinders, u = A r + B / r
    with u(R1) = omega_in R1 and u(R2) = omega_out R2 (the no-slip
    Navier-Stokes solution of Sec. III A)."""
    d = r_out ** 2 - r_in ** 2
    a = (omega_out * r_out ** 2 - omega_in * r_in ** 2) / d
    b = r_in ** 2 * r_out ** 2 * (omega_in - omega_out) / d
    r = np.asarray(r, dtype=np.float64)
    return a * r + b / r


def shock(n_r: int = 2000, n_theta: int = 16, steps: int = 1000, cfl: float = STABLE_CFL,
          tau: float = 2e-5, pressure_ratio: int = 10, r_in: float = 1.0, r_out: float = 3.0,
          r_split: float = 2.0) -> Workload:
    """Radial Riemann problem: (rho, u_r, T) = (1, 0, 1) for r < r_split and
    (0.125, 0, 0.8) beyond (pressure ratio 10), or (0.125, 0, 0.4)
    (pressure ratio 20).  Sharp initial jump; extrapolated walls."""
    R, _ = _mesh(n_r, n_theta, r_in, r_out)
    t_out = {10: 0.8, 20: 0.4}[pressure_ratio]
    inner = R < r_split
    rho = np.where(inner, 1.0, 0.125)
    T = np.where(inner, 1.0, t_out)
    z = np.zeros_like(R)
    dt = dt_from_cfl(cfl, n_r, n_theta, r_in, r_out)
    return Workload(f"shock_pr{pressure_ratio}", n_r, n_theta, r_in, r_out, tau, dt, steps,
                    rho, z.copy(), z.copy(), T, smooth=False,
                    extra={"r_split": r_split, "left": (1.0, 0.0, 1.0), "right": (0.125, 0.0, 0.125 * t_out)})


def _rm_fields(R, TH, r_iface, dr, rho_in=3.0, rho_out=1.0, p0=1.0, r_shock=2.6, mach=2.0,
               width_cells=2.0):
    w = width_cells * dr
    chi = 0.5 * (1.0 - np.tanh((R - r_iface) / w))       # 1 inside, 0 outside
    rho = rho_out + (rho_in - rho_out) * chi
    T = p0 / rho
    u_r = np.zeros_like(R)
    rho_h, u_h, p_h, D = hugoniot_from_mach(rho_out, 0.0, p0, mach, direction=-1.0)
    post = R >= r_shock
    rho = np.where(post, rho_h, rho)
    u_r = np.where(post, u_h, u_r)
    T = np.where(post, p_h / rho_h, T)
    return rho, u_r, np.zeros_like(R), T, (rho_h, u_h, p_h / rho_h, D)


def _rm_bc(n_theta, post):
    rho_h, u_h, t_h, _ = post
    v = np.zeros((2, 4, n_theta))
    v[:, 0, :] = rho_h
    v[:, 1, :] = u_h
    v[:, 2, :] = 0.0
    v[:, 3, :] = t_h
    return (None, v)


def rm(n_r: int = 1024, n_theta: int = 2048, steps: int = 5000, cfl: float = STABLE_CFL,
       tau: float = 1e-5, amp: float = 0.02, mode: int = 8, r_in: float = 1.0,
       r_out: float = 3.0) -> Workload:
    """Richtmyer-Meshkov: interface r = 2 + amp cos(mode theta), heavy inner
    gas (rho 3 vs 1, equal pressure 1), inward Mach-2 shock starting at r=2.6
    with the Rankine-Hugoniot post-shock state (Eq. 45) behind it.  The
    interface is smoothed over 2 dr (tanh).  Inner wall extrapolated, outer
    wall held at the post-shock state.  The CFL-based dt is far above tau;
    runs that follow the shock through the interface need dt of the order
    of tau (the paper's RM runs use dt = tau = 1e-5)."""
    R, TH = _mesh(n_r, n_theta, r_in, r_out)
    dr = (r_out - r_in) / (n_r - 1)
    r_if = 2.0 + amp * np.cos(mode * TH)
    rho, u_r, u_th, T, post = _rm_fields(R, TH, r_if, dr)
    return Workload("rm", n_r, n_theta, r_in, r_out, tau, dt_from_cfl(cfl, n_r, n_theta, r_in, r_out),
                    steps, rho, u_r, u_th, T, bc_kind=(BC_EXTRAP, BC_DIRICHLET),
                    bc_values=_rm_bc(n_theta, post), smooth=False,
                    extra={"post_shock": post})


def rm_amplitudes(seed: int = 20130228, n_modes: int = 16, scale: float = 0.01) -> np.ndarray:
    """Interface mode amplitudes a_k ~ U(0, scale), k = 1..n_modes."""
    return np.random.default_rng(seed).uniform(0.0, scale, size=n_modes)


def rm_background(R, TH, amp: float):
    """Smooth, bounded background modulation 1 + amp s(r, theta) used to keep
    every region of an RM state non-uniform (for finite-difference checks: a
    limiter sitting exactly on its kink has no derivative)."""
    return 1.0 + amp * np.sin(3.0 * TH + 1.7 * R) * np.cos(2.3 * R - TH)


def rm_adj(n_r: int = 512, n_theta: int = 1024, steps: int = 2000, cfl: float = STABLE_CFL,
           tau: float = 1e-5, a: Optional[np.ndarray] = None, seed: int = 20130228,
           r_in: float = 1.0, r_out: float = 3.0, background: float = 0.0,
           dt: Optional[float] = None) -> Workload:
    """RM with interface r = 2 + sum_k a_k cos(k theta), k = 1..16.  A nonzero
    ``background`` multiplies rho and T by rm_background (pressure changes
    slightly; used only by gradient checks).  ``dt`` overrides the CFL-based
    time step (the paper's RM runs use dt = tau)."""
    if a is None:
        a = rm_amplitudes(seed)
    R, TH = _mesh(n_r, n_theta, r_in, r_out)
    dr = (r_out - r_in) / (n_r - 1)
    k = np.arange(1, len(a) + 1, dtype=np.float64)
    r_if = 2.0 + np.tensordot(np.cos(np.multiply.outer(TH, k)), a, axes=([2], [0]))
    rho, u_r, u_th, T, post = _rm_fields(R, TH, r_if, dr)
    if background:
        m = rm_background(R, TH, background)
        rho = rho * m
        T = T * m
    if dt is None:
        dt = dt_from_cfl(cfl, n_r, n_theta, r_in, r_out)
    return Workload("rm_adj", n_r, n_theta, r_in, r_out, tau, dt,
                    steps, rho, u_r, u_th, T, bc_kind=(BC_EXTRAP, BC_DIRICHLET),
                    bc_values=_rm_bc(n_theta, post), smooth=False,
                    extra={"a": np.asarray(a, dtype=np.float64), "seed": seed, "post_shock": post,
                           "background": background})


def kh(n_r: int = 4096, n_theta: int = 4096, steps: int = 10000, cfl: float = STABLE_CFL,
       tau: float = 1e-5, u0: float = 0.5, r_in: float = 1.0, r_out: float = 3.0) -> Workload:
    """Kelvin-Helmholtz: u_theta = u0 tanh((r-2)/0.02),
    u_r = 0.01 sin(16 theta) exp(-((r-2)/0.05)^2), rho = 1.5 + 0.5 tanh((r-2)/0.02)
    (1 inner, 2 outer), uniform pressure 1.  Extrapolated walls."""
    R, TH = _mesh(n_r, n_theta, r_in, r_out)
    s = np.tanh((R - 2.0) / 0.02)
    rho = 1.5 + 0.5 * s
    u_th = u0 * s
    u_r = 0.01 * np.sin(16.0 * TH) * np.exp(-((R - 2.0) / 0.05) ** 2)
    T = 1.0 / rho
    return Workload("kh", n_r, n_theta, r_in, r_out, tau, dt_from_cfl(cfl, n_r, n_theta, r_in, r_out),
                    steps, rho, u_r, u_th, T, extra={"u0": u0})


def uniform(n_r: int, n_theta: int, rho: float = 1.3, ux: float = 0.31, uy: float = -0.17,
            T: float = 0.9, tau: float = 1e-3, cfl: float = 0.5, r_in: float = 1.0,
            r_out: float = 2.0, n_dirs: int = 8, n_f: int = 8) -> Workload:
    """Uniform density and temperature with a uniform *Cartesian* velocity
    (so u_r, u_theta vary with theta).  Extrapolated walls."""
    R, TH = _mesh(n_r, n_theta, r_in, r_out, n_dirs, n_f)
    u_r = ux * np.cos(TH) + uy * np.sin(TH)
    u_th = -ux * np.sin(TH) + uy * np.cos(TH)
    return Workload("uniform", n_r, n_theta, r_in, r_out, tau,
                    dt_from_cfl(cfl, n_r, n_theta, r_in, r_out, n_dirs, n_f), 1,
                    np.full_like(R, rho), u_r, u_th, np.full_like(R, T),
                    n_dirs=n_dirs, n_f=n_f, B=TABLE1_B[n_dirs])


def random_smooth(n_r: int, n_theta: int, seed: int = 1, tau: float = 2e-3, cfl: float = STABLE_CFL,
                  r_in: float = 1.0, r_out: float = 2.0, amp: float = 0.2,
                  bc_kind=(BC_EXTRAP, BC_EXTRAP), n_dirs: int = 8, n_f: int = 8) -> Workload:
    """Smooth random fields: a few low Fourier modes in theta times smooth
    radial profiles, around rho = 1, T = 1, |u| ~ 0.3."""
    rng = np.random.default_rng(seed)
    R, TH = _mesh(n_r, n_theta, r_in, r_out, n_dirs, n_f)
    x = (R - r_in) / (r_out - r_in)
    period = 2.0 * math.pi * n_f / n_dirs

    def field(base, scale):
        out = np.full_like(R, base)
        for m in range(1, 4):
            k = 2.0 * math.pi * m / period
            a, b, c, d = rng.uniform(-1, 1, 4)
            out += scale / m * (a * np.cos(k * TH + b) * np.cos(math.pi * (m * x + c)) + 0.3 * d * x)
        return out

    rho = field(1.0, amp)
    T = field(1.0, amp)
    u_r = field(0.0, 0.3)
    u_th = field(0.1, 0.3)
    vals = []
    for side in range(2):
        v = np.zeros((2, 4, n_theta))
        v[:, 0, :] = 1.0 + 0.05 * side
        v[:, 1, :] = 0.02
        v[:, 2, :] = 0.1 - 0.05 * side
        v[:, 3, :] = 0.95
        vals.append(v)
    return Workload("random_smooth", n_r, n_theta, r_in, r_out, tau,
                    dt_from_cfl(cfl, n_r, n_theta, r_in, r_out, n_dirs, n_f), 1,
                    rho, u_r, u_th, T, bc_kind=tuple(bc_kind), bc_values=tuple(vals),
                    n_dirs=n_dirs, n_f=n_f, B=TABLE1_B[n_dirs])


def by_name(name: str, **kw) -> Workload:
    table = {"rot": rot, "shock": shock, "rm": rm, "rm_adj": rm_adj, "kh": kh,
             "uniform": uniform, "random_smooth": random_smooth}
    return table[name](**kw)
