"""Pins of the oracle's Modified Warming-Beam scheme (Sec. II B 3) against
the properties the paper states for it and against the classical
Warming-Beam scheme it modifies (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O


def _wb(C, pm2, pm1, p0, pp1, pp2):
    """Classical Warming-Beam update, Eq. (25), written out independently."""
    if C >= 0:
        return p0 - C * (p0 - pm1) - 0.5 * C * (1 - C) * (p0 - 2 * pm1 + pm2)
    return p0 - C * (pp1 - p0) + 0.5 * C * (1 + C) * (p0 - 2 * pp1 + pp2)


@pytest.mark.parametrize("C", [0.0, 0.3, 0.77, 1.0, -0.2, -0.9, -1.0, 1.6, -1.4])
def test_mwb_equals_wb_when_switch_vanishes(C):
    # |eta| = 1 gives S(eta) = 0 (Eq. 37), and Eq. (28) collapses to Eq. (26),
    # the rewritten Warming-Beam scheme of Eq. (25).
    rng = np.random.default_rng(3)
    for _ in range(50):
        p0, d = rng.normal(), rng.normal()
        sgn = rng.choice([-1.0, 1.0])     # eta = +1 or -1
        if C >= 0:
            pm1 = p0 - d
            pm2 = pm1 - sgn * d
            pp1, pp2 = rng.normal(size=2)
        else:
            pp1 = p0 + d
            pp2 = pp1 + sgn * d
            pm2, pm1 = rng.normal(size=2)
        got = p0 - O.mwb_increment(C, pm2, pm1, p0, pp1, pp2)
        assert got == pytest.approx(_wb(C, pm2, pm1, p0, pp1, pp2), rel=1e-13, abs=1e-14)


def test_switch_function_closed_form():
    # (1 - S(eta)) (1 - eta) delta with S = (|eta|-1)/(|eta|+1) equals
    # 2 |delta| (delta - delta_up) / (|delta| + |delta_up|) wherever eta is defined.
    rng = np.random.default_rng(5)
    for _ in range(200):
        C = rng.uniform(0.01, 0.99)
        pm2, pm1, p0 = rng.normal(size=3)
        d, du = p0 - pm1, pm1 - pm2
        h = 2 * abs(d) * (d - du) / (abs(d) + abs(du))
        want = C * d + 0.5 * C * (1 - C) * h
        assert O.mwb_increment(C, pm2, pm1, p0, 0.0, 0.0) == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_unit_courant_number_is_an_exact_shift():
    # phi(1) = phi(-1) = 1 (Eq. 31): the scheme translates by one node.
    psi = np.random.default_rng(0).normal(size=40)
    assert np.allclose(O.mwb_1d(psi, 1.0), np.roll(psi, 1), rtol=0, atol=1e-14)
    assert np.allclose(O.mwb_1d(psi, -1.0), np.roll(psi, -1), rtol=0, atol=1e-14)


def test_zero_courant_number_is_identity():
    psi = np.random.default_rng(1).normal(size=17)
    assert np.array_equal(O.mwb_1d(psi, 0.0), psi)


def test_flat_profile_is_unchanged():
    psi = np.full(12, 0.37)
    for C in (0.4, -0.6, 1.0):
        assert np.array_equal(O.mwb_1d(psi, C), psi)


@pytest.mark.parametrize("C", [0.05, 0.25, 0.5, 0.9, 1.0, -0.3, -0.8])
def test_new_value_is_a_convex_combination(C):
    # 0 <= phi(C) <= 1 (Eqs. 29-37): psi_j^{n+1} lies between psi_j and its
    # upwind neighbour, so no new extrema appear, for any data.
    rng = np.random.default_rng(11)
    for _ in range(20):
        psi = rng.normal(size=30) * rng.uniform(0.1, 10)
        out = O.mwb_1d(psi, C)
        up = np.roll(psi, 1 if C >= 0 else -1)
        lo, hi = np.minimum(psi, up), np.maximum(psi, up)
        tol = 1e-13 * np.max(np.abs(psi))
        assert np.all(out >= lo - tol) and np.all(out <= hi + tol)


def test_step_profile_no_overshoot_while_wb_overshoots():
    psi = np.where(np.arange(60) < 30, 1.0, 0.0)
    C = 0.5
    m, w = psi.copy(), psi.copy()
    n = len(psi)
    for _ in range(20):
        m = O.mwb_1d(m, C)
        w = np.array([_wb(C, w[(j - 2) % n], w[(j - 1) % n], w[j], w[(j + 1) % n], w[(j + 2) % n])
                      for j in range(n)])
    assert m.max() <= 1.0 + 1e-14 and m.min() >= -1e-14
    assert w.max() > 1.01 or w.min() < -0.01


def test_smooth_translation_converges():
    # Advection of a smooth periodic pulse to t = 1 at C = 0.5: the error
    # shrinks under refinement (the scheme is consistent).
    errs = []
    for n in (50, 100, 200, 400):
        x = np.arange(n) / n
        psi = np.exp(-((x - 0.5) / 0.1) ** 2)
        C = 0.5
        steps = int(round(0.25 * n / C))      # move by a quarter period
        for _ in range(steps):
            psi = O.mwb_1d(psi, C)
        exact = np.exp(-(((x - 0.25 - 0.5 + 0.5) % 1.0 - 0.5) / 0.1) ** 2)
        errs.append(np.abs(psi - exact).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert orders[-1] > 0.9, (errs, orders)


def test_removable_singularity_at_zero_delta():
    # delta = 0 with a nonzero upstream difference: the bracket is undefined but
    # its product with delta tends to 0; h -> 0 as well.
    assert O.mwb_increment(0.4, 0.0, 1.0, 1.0, 5.0, 7.0) == 0.0
    assert O.mwb_increment(-0.4, 3.0, 2.0, 1.0, 1.0, 9.0) == 0.0
    tiny = 1e-300
    got = O.mwb_increment(0.4, -1.0, 1.0, 1.0 + tiny, 0.0, 0.0)
    assert abs(got) < 1e-299
