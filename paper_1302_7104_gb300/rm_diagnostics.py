"""Richtmyer-Meshkov interface diagnostics (Sec. III C).

Post-processing of the fields the library returns (pclb_moments): the radius
of the material interface in every azimuthal row, its amplitude (half the
crest-to-trough distance) and mean position, and the theory the paper
compares them with:

* the one-dimensional shock-interface interaction (an exact Riemann problem
  for the ideal gas with gamma = 2): the interface velocity change du, the
  post-shock Atwood number A_t and the compression ratio Cmpr = 1 - du / D
  of an interface hit by a shock of speed D;
* Richtmyer's impulsive model, dA/dt = k du A_t A_1 with A_1 = A_0 Cmpr;
* the Zhang-Sohn nonlinear model,
  dA/dt = v0 / (1 + zeta k^2 v0 A_1 t + max[0, (k A_1)^2 - A_t^2 + 0.5] (k v0 t)^2),
  v0 = k du A_t A_1, zeta = +1 light to heavy, -1 heavy to light.

The interface is located as the contact between the two materials: where
the entropy variable s = ln(p / rho^gamma) crosses the mean of the two
materials' values (shocks change s little, the contact separates the gases'
very different s; density alone would also flag the shocks).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from .inputs import GAMMA, hugoniot_from_speed


# ---------------------------------------------------------------------------
# exact Riemann problem (pressure function bracketed and bisected)
# ---------------------------------------------------------------------------
def _wave_velocity_jump(p: float, rho: float, pk: float, g: float) -> float:
    """Velocity change across a left- or right-facing wave that takes the
    state (rho, pk) to pressure p: shock for p > pk, rarefaction otherwise."""
    if p > pk:
        a = 2.0 / ((g + 1.0) * rho)
        b = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * math.sqrt(a / (p + b))
    c = math.sqrt(g * pk / rho)
    return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(left: Sequence[float], right: Sequence[float], gamma: float = GAMMA):
    """Pressure and velocity (p*, u*) between the two waves of the Riemann
    problem with the states left = (rho, u, p) and right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    fun = lambda p: _wave_velocity_jump(p, rl, pl, gamma) + _wave_velocity_jump(p, rr, pr, gamma) + (ur - ul)
    lo, hi = 1e-14, max(pl, pr)
    while fun(hi) < 0.0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if fun(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    p = 0.5 * (lo + hi)
    u = 0.5 * (ul + ur) + 0.5 * (_wave_velocity_jump(p, rr, pr, gamma) - _wave_velocity_jump(p, rl, pl, gamma))
    return p, u


def _density_behind(p: float, rho: float, pk: float, g: float) -> float:
    """Density of (rho, pk) after a shock (p > pk) or isentrope to p."""
    if p > pk:
        r = p / pk
        return rho * (r + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * r + 1.0)
    return rho * (p / pk) ** (1.0 / g)


def shock_interface(pre_a: Sequence[float], D: float, pre_b: Sequence[float], gamma: float = GAMMA) -> dict:
    """A shock of lab-frame speed D (> 0 outward, < 0 inward) runs through gas a
    (rho, u, p) into a material interface with gas b (rho, u, p), both at rest
    initially.  Returns the interface velocity change du (signed), the
    compression ratio 1 - du / D, the post-shock Atwood number
    (rho*_b - rho*_a) / (rho*_b + rho*_a) and the star state."""
    shocked = hugoniot_from_speed(*pre_a, D)
    if D > 0:   # a inside, b outside: left = shocked a
        p, u = star_state(shocked, pre_b, gamma)
    else:       # a outside, b inside: left = b
        p, u = star_state(pre_b, shocked, gamma)
    du = u - pre_b[1]
    rho_a = _density_behind(p, shocked[0], shocked[2], gamma)
    rho_b = _density_behind(p, pre_b[0], pre_b[2], gamma)
    return {"du": du, "compression": 1.0 - du / D, "atwood": (rho_b - rho_a) / (rho_b + rho_a),
            "p_star": p, "u_star": u, "rho_star_a": rho_a, "rho_star_b": rho_b, "shocked_a": shocked}


def richtmyer_rate(k: float, du: float, atwood: float, a0: float, compression: float) -> float:
    """Impulsive model: dA/dt = k du A_t A_1, A_1 = A_0 Cmpr."""
    return k * du * atwood * a0 * compression


def zhang_sohn_rate(t, k: float, du: float, atwood: float, a1: float, zeta: float):
    """Nonlinear model of Zhang and Sohn for the growth rate at time t after
    the shock passage (zeta = +1 light to heavy, -1 heavy to light)."""
    t = np.asarray(t, dtype=np.float64)
    v0 = k * du * atwood * a1
    c2 = max(0.0, (k * a1) ** 2 - atwood ** 2 + 0.5)
    return v0 / (1.0 + zeta * k * k * v0 * a1 * t + c2 * (k * v0 * t) ** 2)


# ---------------------------------------------------------------------------
# interface tracking
# ---------------------------------------------------------------------------
def entropy(rho: np.ndarray, T: np.ndarray, gamma: float = GAMMA) -> np.ndarray:
    """s = ln(p / rho^gamma) with p = rho T."""
    return np.log(T) - (gamma - 1.0) * np.log(rho)


def interface_radii(rho: np.ndarray, T: np.ndarray, r: np.ndarray, r_lo: float, r_hi: float,
                    s_inner: float, s_outer: float, gamma: float = GAMMA) -> np.ndarray:
    """Radius of the contact in every azimuthal row: the first crossing, going
    outward from r_lo, of the entropy level (s_inner + s_outer) / 2, linearly
    interpolated between nodes; NaN where no crossing lies in [r_lo, r_hi].
    rho, T: [n_theta][n_r]; s_inner, s_outer: entropy of the inner and the
    outer material."""
    s = entropy(np.asarray(rho, dtype=np.float64), np.asarray(T, dtype=np.float64), gamma)
    r = np.asarray(r, dtype=np.float64)
    band = np.nonzero((r >= r_lo) & (r <= r_hi))[0]
    i0, i1 = band[0], band[-1]
    level = 0.5 * (s_inner + s_outer)
    sign = 1.0 if s_outer > s_inner else -1.0
    x = sign * (s[:, i0:i1 + 1] - level)          # crosses from < 0 to >= 0
    out = np.full(s.shape[0], np.nan)
    for j in range(s.shape[0]):
        hit = np.nonzero((x[j, :-1] < 0.0) & (x[j, 1:] >= 0.0))[0]
        if len(hit) == 0:
            continue
        m = hit[0]
        a, b = x[j, m], x[j, m + 1]
        out[j] = r[i0 + m] + (r[i0 + m + 1] - r[i0 + m]) * (-a / (b - a))
    return out


def amplitude(radii: np.ndarray) -> float:
    """Half the crest-to-trough distance of the interface."""
    return 0.5 * (np.nanmax(radii) - np.nanmin(radii))
