"""Exact solution of the 1-D Riemann problem for an ideal gas (test helper).

Standard two-wave construction (e.g. Toro, "Riemann Solvers and Numerical
Methods for Fluid Dynamics", ch. 4): Newton iteration on the star-region
pressure, then self-similar sampling at xi = x / t.  Used only to pin the
oracle's shock-tube behaviour; the default ratio gamma = 2 is the paper's.
"""
import math

import numpy as np


def _f_and_df(p, rho, pk, g):
    c = math.sqrt(g * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    e = (g - 1.0) / (2.0 * g)  # rarefaction
    return 2.0 * c / (g - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * c)


def star_state(left, right, g=2.0):
    """left/right = (rho, u, p).  Returns (p_star, u_star)."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-10, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _f_and_df(p, rl, pl, g)
        fr, dr = _f_and_df(p, rr, pr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        p_new = max(1e-12, p - dp)
        if abs(p_new - p) <= 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _f_and_df(p, rl, pl, g)
    fr, _ = _f_and_df(p, rr, pr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, xi, g=2.0):
    """(rho, u, p) at the similarity coordinates xi (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(np.asarray(xi, dtype=np.float64)):
        if s <= us:  # left of the contact
            if ps > pl:
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    w = (rl, ul, pl)
                else:
                    r = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
                    w = (r, us, ps)
            else:
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - cl:
                    w = (rl, ul, pl)
                elif s >= us - cs:
                    w = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    r = rl * (c / cl) ** (2 / (g - 1))
                    w = (r, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:  # right of the contact
            if ps > pr:
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    w = (rr, ur, pr)
                else:
                    r = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
                    w = (r, us, ps)
            else:
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + cr:
                    w = (rr, ur, pr)
                elif s <= us + cs:
                    w = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    r = rr * (c / cr) ** (2 / (g - 1))
                    w = (r, u, pr * (c / cr) ** (2 * g / (g - 1)))
        out[:, n] = w
    return out
