"""Pins of the convection schemes and the relaxation variant the paper compares
(Sec. II B 2-3, Fig. 5): Warming-Beam (Eq. 25), Lax-Wendroff, second-order
upwind and the forward-Euler relaxation (Eq. 18), beside the default MWB and
analytic relaxation (no GPU).

Each scheme advects ψ_t + a ψ_ξ = 0 by ψ_j^{n+1} = ψ_j^n − M_j with the
Courant number C = a Δt / Δξ.  Linear data are translated exactly by all of
them; quadratic data exactly by the two schemes that keep the whole
second-order Taylor term (WB, LW), while the second-order upwind scheme, a
forward-Euler step, misses exactly the C² term; the C < 0 branches are the
mirror images of the C > 0 ones."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I

SCHEMES = (O.SCHEME_MWB, O.SCHEME_WB, O.SCHEME_LW, O.SCHEME_UPWIND2)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("C", [0.3, -0.45, 0.9])
def test_linear_data_are_translated_exactly(scheme, C):
    alpha, j = 0.7, 5
    psi = [alpha * (j + k) for k in (-2, -1, 0, 1, 2)]
    assert O.scheme_increment(scheme, C, *psi) == pytest.approx(C * alpha, rel=1e-13)


@pytest.mark.parametrize("C", [0.25, -0.6])
def test_quadratic_data(C):
    j = 7
    psi = [float((j + k) ** 2) for k in (-2, -1, 0, 1, 2)]
    exact = 2 * C * j - C * C                         # (j - C)^2 = j^2 - M
    assert O.scheme_increment(O.SCHEME_WB, C, *psi) == pytest.approx(exact, rel=1e-13)
    assert O.scheme_increment(O.SCHEME_LW, C, *psi) == pytest.approx(exact, rel=1e-13)
    assert O.scheme_increment(O.SCHEME_UPWIND2, C, *psi) == pytest.approx(2 * C * j, rel=1e-13)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_negative_courant_numbers_mirror_positive_ones(scheme):
    rng = np.random.default_rng(3)
    for _ in range(20):
        psi = rng.normal(size=5)
        C = rng.uniform(0.05, 0.95)
        assert O.scheme_increment(scheme, -C, *psi[::-1]) == pytest.approx(
            O.scheme_increment(scheme, C, *psi), rel=1e-12, abs=1e-15)


def test_mwb_equals_wb_when_the_ratio_has_unit_modulus():
    # eta = (psi_{j-1} - psi_{j-2}) / (psi_j - psi_{j-1}) = 1: S = 0, MWB reduces to WB
    psi = [1.0, 2.0, 3.0, 3.5, 9.0]
    for C in (0.2, 0.7):
        assert O.scheme_increment(O.SCHEME_MWB, C, *psi) == pytest.approx(O.scheme_increment(O.SCHEME_WB, C, *psi))


def _advect_ring(scheme, psi, C):
    """One step of a scheme on a periodic 1-D ring."""
    n = len(psi)
    at = lambda k: psi[k % n]
    return np.array([psi[j] - O.scheme_increment(scheme, C, at(j - 2), at(j - 1), at(j), at(j + 1), at(j + 2))
                     for j in range(n)])


def test_wb_and_lw_overshoot_a_step_while_mwb_does_not():
    step = np.where(np.arange(24) < 12, 1.0, 0.0)
    for C in (0.3, 0.6, -0.4):
        mwb = _advect_ring(O.SCHEME_MWB, step, C)
        assert mwb.min() >= -1e-15 and mwb.max() <= 1.0 + 1e-15
        for s in (O.SCHEME_WB, O.SCHEME_LW, O.SCHEME_UPWIND2):
            out = _advect_ring(s, step, C)
            assert out.min() < -1e-3 or out.max() > 1.0 + 1e-3, (s, C)


def _uniform_noneq(seed):
    """f identical at every node: a uniform Cartesian state plus one departure
    vector, with ghost nodes that carry the departure too, so that every
    convection increment vanishes."""
    w = I.uniform(6, 5)
    w.bc_kind = (I.BC_EXTRAP | I.BC_NEQ, I.BC_EXTRAP | I.BC_NEQ)
    feq = O.set_state(w)
    pert = 1.0 + 0.03 * np.random.default_rng(seed).normal(size=(feq.shape[0], 1, 1))
    return w, feq, np.ascontiguousarray(feq * pert)


def test_forward_euler_relaxation_of_a_uniform_state():
    w, _, f = _uniform_noneq(4)
    feq = O.set_state(w, *O.fields(w, f))              # equilibrium of f's own moments
    for relax, decay in ((O.RELAX_EXACT, np.exp(-w.dt / w.tau)), (O.RELAX_EULER, 1.0 - w.dt / w.tau)):
        w.relaxation = relax
        got = O.step(w, f)
        want = feq + (f - feq) * decay
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(f)), relax


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("relax", [O.RELAX_EXACT, O.RELAX_EULER])
def test_uniform_state_keeps_its_moments(scheme, relax):
    w, _, f = _uniform_noneq(5)
    w.scheme, w.relaxation = scheme, relax
    a = O.fields(w, f)
    b = O.fields(w, O.step(w, f))
    for x, y in zip(a, b):
        assert np.max(np.abs(x - y)) <= 1e-12


def test_schemes_agree_to_second_order_on_smooth_data():
    # one step of each scheme on smooth data: they differ by O(C dx^2) terms only
    w = I.random_smooth(40, 24, seed=6)
    f = O.set_state(w)
    ref = O.step(w, f)
    for s in (O.SCHEME_WB, O.SCHEME_LW):
        w.scheme = s
        d = np.max(np.abs(O.step(w, f) - ref)) / np.max(np.abs(ref))
        assert 0.0 < d < 1e-2, s
    w.scheme = O.SCHEME_MWB
