"""Pins of the RM interface diagnostics (Sec. III C; no GPU): the
shock-interface theory against the compression ratios the paper prints and
against an independent exact Riemann solver, the growth-rate models against
each other, and the interface tracker on a field with a known interface."""
import math
import os

import numpy as np
import pytest

import riemann_exact as RE
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import rm_diagnostics as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rm_compression_theory.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        label, D, rho_b, cmpr, digits = line.split()
        rows.append((label, float(D), float(rho_b), float(cmpr), int(digits)))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: r[0])
def test_compression_ratio_matches_the_printed_theory(row):
    _, D, rho_b, cmpr, digits = row
    got = R.shock_interface((1.0, 0.0, 1.0), D, (rho_b, 0.0, 1.0))["compression"]
    # the printed value carries `digits` decimals; one more unit of slack for its rounding
    assert abs(got - cmpr) <= 3 * 10.0 ** (-digits)


def test_star_state_matches_the_reference_solver():
    rng = np.random.default_rng(1)
    for _ in range(30):
        left = (rng.uniform(0.2, 3), rng.uniform(-1, 1), rng.uniform(0.2, 5))
        right = (rng.uniform(0.2, 3), rng.uniform(-1, 1), rng.uniform(0.2, 5))
        p, u = R.star_state(left, right)
        p2, u2 = RE.star_state(left, right)
        assert p == pytest.approx(p2, rel=1e-10) and u == pytest.approx(u2, rel=1e-9, abs=1e-12)


def test_inward_and_outward_shocks_are_mirror_images():
    out = R.shock_interface((1.0, 0.0, 1.0), 2.0, (3.0, 0.0, 1.0))
    inw = R.shock_interface((1.0, 0.0, 1.0), -2.0, (3.0, 0.0, 1.0))
    assert inw["du"] == pytest.approx(-out["du"]) and inw["compression"] == pytest.approx(out["compression"])
    assert inw["atwood"] == pytest.approx(out["atwood"])
    assert out["atwood"] > 0 > R.shock_interface((1.0, 0.0, 1.0), 2.0, (0.5, 0.0, 1.0))["atwood"]


def test_growth_models_agree_at_shock_passage():
    th = R.shock_interface((1.0, 0.0, 1.0), 2.0, (3.0, 0.0, 1.0))
    k, a0 = 20.0, 0.02
    v_r = R.richtmyer_rate(k, th["du"], th["atwood"], a0, th["compression"])
    a1 = a0 * th["compression"]
    zs = R.zhang_sohn_rate(np.array([0.0, 0.05, 0.2]), k, th["du"], th["atwood"], a1, zeta=1.0)
    assert zs[0] == pytest.approx(v_r)
    assert zs[0] > zs[1] > zs[2] > 0                  # the nonlinear model saturates


def test_tracker_recovers_a_known_interface():
    n_r, n_t = 400, 256
    r = I.radii(n_r, 1.0, 3.0)
    th = I.angles(n_t)
    R_, TH = np.meshgrid(r, th)
    a0, m = 0.02, 8
    r_if = 2.0 + a0 * np.cos(m * TH)
    chi = 0.5 * (1.0 - np.tanh((R_ - r_if) / (2 * (r[1] - r[0]))))
    rho = 1.0 + 2.0 * chi
    T = 1.0 / rho                                      # equal pressure
    s_in, s_out = math.log(1 / 3) - math.log(3), 0.0
    radii = R.interface_radii(rho, T, r, 1.5, 2.5, s_in, s_out)
    assert not np.any(np.isnan(radii))
    assert R.amplitude(radii) == pytest.approx(a0, rel=0.02)
    # the entropy midpoint sits where rho is the geometric mean of the two
    # densities, half a node from the centre of the tanh profile
    assert np.mean(radii) == pytest.approx(2.0, abs=r[1] - r[0])
