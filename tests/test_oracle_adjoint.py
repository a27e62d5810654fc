"""Pins of the oracle's adjoint step (the vector-Jacobian product of one
combined-scheme step) against central finite differences of the oracle's
forward step and against the dot-product identity (no GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I


def _state(n_r=6, n_t=8, seed=3, bc=(I.BC_EXTRAP, I.BC_EXTRAP)):
    w = I.random_smooth(n_r, n_t, seed=seed, bc_kind=bc)
    f = O.set_state(w)
    # a non-equilibrium part so that the relaxation's Jacobian matters
    rng = np.random.default_rng(seed + 100)
    f = f * (1.0 + 0.02 * rng.normal(size=f.shape))
    return w, f


@pytest.mark.parametrize("bc", [(I.BC_EXTRAP, I.BC_EXTRAP), (I.BC_DIRICHLET, I.BC_WALL),
                                (I.BC_EXTRAP | I.BC_NEQ, I.BC_WALL | I.BC_NEQ)])
def test_jvp_matches_central_differences(bc):
    w, f = _state(bc=bc)
    rng = np.random.default_rng(0)
    df = rng.normal(size=f.shape) * np.abs(f).max()
    jv = O.step_jvp(w, f, df)
    # The switch function has large curvature where differences are small, so
    # the central difference converges like eps^2 from a large constant.
    scale = np.max(np.abs(jv))
    for eps, tol in ((1e-7, 2e-5), (1e-8, 1e-6)):
        fd = (O.step(w, f + eps * df) - O.step(w, f - eps * df)) / (2 * eps)
        assert np.max(np.abs(fd - jv)) <= tol * scale, eps


def test_adjoint_is_the_transpose_of_the_jvp():
    w, f = _state(n_r=5, n_t=6)
    rng = np.random.default_rng(1)
    lam = rng.normal(size=f.shape)
    adj = O.adjoint_step(w, f, lam)
    for _ in range(3):
        df = rng.normal(size=f.shape)
        lhs = np.sum(lam * O.step_jvp(w, f, df))
        rhs = np.sum(adj * df)
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12 * np.abs(lhs).max())


@pytest.mark.parametrize("bc", [(I.BC_EXTRAP, I.BC_EXTRAP), (I.BC_DIRICHLET | I.BC_NEQ, I.BC_EXTRAP | I.BC_NEQ)])
def test_adjoint_matches_finite_difference_gradient(bc):
    # d/d f_j of <lam, step(f)> by central differences on a few entries,
    # including entries next to the walls (ghost extrapolation feeds back;
    # non-equilibrium ghosts also carry the wall node's own f - f^eq, Sec. II C)
    w, f = _state(n_r=5, n_t=6, seed=8, bc=bc)
    rng = np.random.default_rng(2)
    lam = rng.normal(size=f.shape)
    adj = O.adjoint_step(w, f, lam)
    picks = [(0, 0, 0), (5, 2, 0), (12, 3, 1), (20, 5, 4), (32, 1, 2), (17, 0, 3)]
    for idx in picks:
        e = np.zeros_like(f)
        e[idx] = 1.0
        h = 1e-6 * max(1.0, abs(f[idx]))
        fd = (np.sum(lam * O.step(w, f + h * e)) - np.sum(lam * O.step(w, f - h * e))) / (2 * h)
        assert adj[idx] == pytest.approx(fd, rel=1e-6, abs=1e-8), idx


def test_adjoint_of_complete_relaxation_conserves_moment_weights():
    # dt -> 0 with dt / tau large: the convection Courant numbers vanish and the
    # step is f -> f^eq(m(f)).  f^eq has the moments of f (Eqs. 3-5), so for a
    # collision invariant psi (1, v_x, v_y, |v|^2/2) the adjoint maps psi to itself.
    w = I.uniform(7, 8)
    w.dt, w.tau = 1e-13, 1e-15
    rng = np.random.default_rng(4)
    fq = O.feq(1.1, 0.2, -0.1, 0.9, 8, I.SPEEDS, I.TABLE1_B[8])
    f = np.ascontiguousarray(np.broadcast_to(fq[:, None, None], (33, 8, 7)))
    f = f * (1 + 0.03 * rng.normal(size=f.shape))
    vx, vy, _ = O.dvm()
    for weight in (np.ones(33), vx, vy, 0.5 * (vx * vx + vy * vy)):
        lam = np.ascontiguousarray(np.broadcast_to(weight[:, None, None], f.shape))
        adj = O.adjoint_step(w, f, lam)
        assert np.max(np.abs(adj - lam)) <= 1e-9 * np.abs(weight).max()
    # a non-invariant weight is not preserved
    lam = np.zeros_like(f)
    lam[9] = 1.0
    assert np.max(np.abs(O.adjoint_step(w, f, lam) - lam)) > 1e-3


def test_set_state_jvp_matches_central_differences():
    w = I.random_smooth(7, 6, seed=12)
    fields = [np.array(x) for x in w.fields()]
    rng = np.random.default_rng(5)
    dfields = [rng.normal(size=x.shape) * 0.1 for x in fields]
    jv = O.set_state_jvp(w, fields, dfields)
    eps = 1e-6

    def at(sign):
        return O.set_state(w, *[x + sign * eps * d for x, d in zip(fields, dfields)])

    fd = (at(1) - at(-1)) / (2 * eps)
    assert np.max(np.abs(fd - jv)) <= 1e-7 * np.max(np.abs(jv))


def test_fields_jvp_matches_central_differences():
    w = I.random_smooth(7, 6, seed=13)
    f = O.set_state(w)
    rng = np.random.default_rng(6)
    df = rng.normal(size=f.shape) * 0.01
    jv = O.fields_jvp(w, f, df)
    eps = 1e-6
    plus, minus = O.fields(w, f + eps * df), O.fields(w, f - eps * df)
    for a, b, j in zip(plus, minus, jv):
        assert np.max(np.abs((a - b) / (2 * eps) - j)) <= 1e-7 * max(np.max(np.abs(j)), 1e-12)

