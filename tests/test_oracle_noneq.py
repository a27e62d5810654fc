"""Pins of the oracle's non-equilibrium manifestations (Sec. IV): the moments
M_2, M_3, M_{3,1}, M_{4,2} and their central counterparts, and the departures
Delta_m, Delta*_m (no GPU).

At equilibrium the moments must equal the relations the discrete velocity
model is built to satisfy (Eqs. 6-9, the fourth-order one in its corrected
form), the central moments those of a Maxwellian (rho E I, 0, 0, 2 rho E^2 I)
and both departures must vanish.  Away from equilibrium the departures obey
identities that follow from mass, momentum and energy conservation of the
collision, which fix the central departures in terms of the plain ones."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I

C = {name: i for i, name in enumerate(O.NEQ_COMPONENTS)}


def _eq_state(seed=3):
    w = I.random_smooth(6, 9, seed=seed)
    rho, ur, ut, T = [np.asarray(x, dtype=np.float64) for x in w.fields()]
    return w, O.set_state(w), rho, ur, ut, T   # gamma = 2: E = T


def test_equilibrium_moments_match_the_model_relations():
    w, f, rho, ur, ut, E = _eq_state()
    M = O.noneq(w, f, O.NEQ_M)[0]
    u2 = ur * ur + ut * ut
    want = {
        "2rr": rho * (E + ur * ur), "2rt": rho * ur * ut, "2tt": rho * (E + ut * ut),
        "3rrr": rho * (3 * E * ur + ur ** 3), "3rrt": rho * (E * ut + ur * ur * ut),
        "3rtt": rho * (E * ur + ur * ut * ut), "3ttt": rho * (3 * E * ut + ut ** 3),
        "31r": rho * ur * (2 * E + 0.5 * u2), "31t": rho * ut * (2 * E + 0.5 * u2),
        "42rr": rho * ((2 * E + 0.5 * u2) * E + (3 * E + 0.5 * u2) * ur * ur),
        "42rt": rho * (3 * E + 0.5 * u2) * ur * ut,
        "42tt": rho * ((2 * E + 0.5 * u2) * E + (3 * E + 0.5 * u2) * ut * ut),
    }
    for name, ref in want.items():
        assert np.max(np.abs(M[C[name]] - ref)) <= 1e-12 * np.max(np.abs(M)), name


def test_equilibrium_central_moments_are_maxwellian():
    w, f, rho, ur, ut, E = _eq_state(4)
    Ms = O.noneq(w, f, O.NEQ_MSTAR)[0]
    scale = np.max(np.abs(Ms))
    want = {"2rr": rho * E, "2tt": rho * E, "42rr": 2 * rho * E * E, "42tt": 2 * rho * E * E}
    for name in O.NEQ_COMPONENTS:
        ref = want.get(name, np.zeros_like(rho))
        assert np.max(np.abs(Ms[C[name]] - ref)) <= 1e-12 * scale, name


def test_departures_vanish_at_equilibrium():
    w, f, *_ = _eq_state(5)
    out = O.noneq(w, f, O.NEQ_M | O.NEQ_DELTA | O.NEQ_MSTAR | O.NEQ_DSTAR)
    assert out.shape == (4, 12, w.n_theta, w.n_r)
    scale = np.max(np.abs(out[0]))
    assert np.max(np.abs(out[1])) <= 1e-13 * scale
    assert np.max(np.abs(out[3])) <= 1e-13 * scale


def _noisy(seed):
    w = I.random_smooth(5, 8, seed=seed)
    f = O.set_state(w)
    f = f * (1.0 + 0.05 * np.random.default_rng(seed).normal(size=f.shape))
    rho, ur, ut, E = O.fields(w, f)
    return w, f, ur, ut


def test_departures_obey_the_conservation_identities():
    w, f, ur, ut = _noisy(7)
    D, Ds = O.noneq(w, f, O.NEQ_DELTA | O.NEQ_DSTAR)
    d = {k: D[C[k]] for k in C}
    ds = {k: Ds[C[k]] for k in C}
    scale = np.max(np.abs(D))
    assert scale > 1e-3                        # really away from equilibrium
    tol = 1e-12 * scale
    # energy is conserved: the trace of Delta_2 vanishes
    assert np.max(np.abs(d["2rr"] + d["2tt"])) <= tol
    # mass and momentum are conserved: the central second-order departure is the plain one
    for k in ("2rr", "2rt", "2tt"):
        assert np.max(np.abs(ds[k] - d[k])) <= tol, k
    # third order: Delta*_abc = Delta_abc - u_a Delta_bc - u_b Delta_ac - u_c Delta_ab
    want = {
        "3rrr": d["3rrr"] - 3 * ur * d["2rr"],
        "3rrt": d["3rrt"] - 2 * ur * d["2rt"] - ut * d["2rr"],
        "3rtt": d["3rtt"] - ur * d["2tt"] - 2 * ut * d["2rt"],
        "3ttt": d["3ttt"] - 3 * ut * d["2tt"],
        # contracted: Delta*_{3,1} = Delta_{3,1} - Delta_2 . u (trace of Delta_2 is 0)
        "31r": d["31r"] - (d["2rr"] * ur + d["2rt"] * ut),
        "31t": d["31t"] - (d["2rt"] * ur + d["2tt"] * ut),
    }
    for k, ref in want.items():
        assert np.max(np.abs(ds[k] - ref)) <= 1e-11 * scale, k


def test_plain_moments_split_into_equilibrium_and_departure():
    # M_m(f) - Delta_m = M_m(f^eq) must equal the closed forms at the moments of f
    w, f, ur, ut = _noisy(8)
    rho, ur, ut, E = O.fields(w, f)
    M, D = O.noneq(w, f, O.NEQ_M | O.NEQ_DELTA)
    Meq = M - D
    u2 = ur * ur + ut * ut
    scale = np.max(np.abs(M))
    assert np.max(np.abs(Meq[C["2rr"]] - rho * (E + ur * ur))) <= 1e-12 * scale
    assert np.max(np.abs(Meq[C["42rt"]] - rho * (3 * E + 0.5 * u2) * ur * ut)) <= 1e-12 * scale
    assert np.max(np.abs(Meq[C["3rrt"]] - rho * (E * ut + ur * ur * ut))) <= 1e-12 * scale


def test_noneq_rejects_bad_groups():
    w, f, *_ = _eq_state()
    with pytest.raises(ValueError):
        O.noneq(w, f, 0)
    with pytest.raises(ValueError):
        O.noneq(w, f, 16)
