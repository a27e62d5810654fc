"""Pins of the oracle's node-sampled step and adjoint entries (used for the
full-size sampled parity checks) against the oracle's whole-grid step and
whole-grid adjoint, on small grids (no GPU).

The sampled step forms the ghost values of Sec. II C (Eqs. 39, 40) on demand
instead of for the whole grid, with the same operations, so it must agree
with the whole-grid step bit for bit; the sampled adjoint restricts the
forward-mode sweep of each entry to the nodes whose update can read it, so it
must agree with the whole-grid adjoint (every output swept) to rounding."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I


def _noisy(w, seed):
    f = O.set_state(w)
    rng = np.random.default_rng(seed)
    return f * (1.0 + 0.02 * rng.normal(size=f.shape))


CASES = [
    ("extrap", lambda: I.random_smooth(7, 9, seed=1, bc_kind=(I.BC_EXTRAP, I.BC_EXTRAP))),
    ("dirichlet_wall", lambda: I.random_smooth(6, 5, seed=2, bc_kind=(I.BC_DIRICHLET, I.BC_WALL))),
    ("rot", lambda: I.rot(n_r=8, n_theta=12)),
    ("rm", lambda: I.rm(n_r=16, n_theta=8)),
    ("sector", lambda: I.random_smooth(6, 5, seed=4, n_f=1)),
    ("three_rows", lambda: I.random_smooth(5, 3, seed=5)),
    # non-equilibrium ghosts: the ghosts also carry the wall node's f - f^eq
    ("neq_extrap_wall", lambda: I.random_smooth(6, 5, seed=6, bc_kind=(I.BC_EXTRAP | I.BC_NEQ, I.BC_WALL | I.BC_NEQ))),
    ("neq_wall_dirichlet", lambda: I.random_smooth(5, 6, seed=7, bc_kind=(I.BC_WALL, I.BC_DIRICHLET | I.BC_NEQ))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_step_nodes_equals_whole_grid_step(name, make):
    w = make()
    f = _noisy(w, 10)
    full = O.step(w, f)
    it, ir = np.meshgrid(np.arange(w.n_theta), np.arange(w.n_r), indexing="ij")
    it, ir = it.ravel(), ir.ravel()
    perm = np.random.default_rng(0).permutation(len(it))     # order of the nodes must not matter
    got = O.step_nodes(w, f, it[perm], ir[perm])
    want = full[:, it[perm], ir[perm]].T
    assert np.array_equal(got, want)


@pytest.mark.parametrize("name,make", CASES[:2] + CASES[4:], ids=[c[0] for c in CASES[:2] + CASES[4:]])
def test_adjoint_entries_equal_whole_grid_adjoint(name, make):
    w = make()
    if w.n_r * w.n_theta > 40:
        w = I.random_smooth(5, 6, seed=3, bc_kind=w.bc_kind, n_f=w.n_f) if w.bc_kind[0] == I.BC_EXTRAP else \
            I.random_smooth(5, 6, seed=3, bc_kind=w.bc_kind)
    f = _noisy(w, 11)
    lam = np.random.default_rng(12).normal(size=f.shape)
    whole = O.adjoint_step(w, f, lam)
    Q = whole.shape[0]
    q, it, ir = np.meshgrid(np.arange(Q), np.arange(w.n_theta), np.arange(w.n_r), indexing="ij")
    got = O.adjoint_entries(w, f, lam, q.ravel(), it.ravel(), ir.ravel())
    want = whole.ravel()
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-13 * scale


def test_sampled_calls_reject_out_of_range_nodes():
    w = I.random_smooth(5, 4, seed=6)
    f = O.set_state(w)
    with pytest.raises(ValueError):
        O.step_nodes(w, f, [4], [0])
    with pytest.raises(ValueError):
        O.adjoint_entries(w, f, f, [33], [0], [0])
