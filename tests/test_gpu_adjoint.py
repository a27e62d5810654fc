"""The GPU adjoint step and the field VJPs against the oracle (GPU).

FP64: the adjoint step equals the oracle's vector-Jacobian product (built
column by column from forward-mode derivatives of the oracle's step) within
1e-12 of its largest entry; on multi-tile grids (ragged tails, walls of every
kind, sectors) every entry equals the oracle's entry computed on its own
(``oracle.adjoint_entries``), and the transpose identity
<lam, J df> = <J^T lam, df> holds against the oracle's JVP.  FP32: within
1e-4.  The field VJPs satisfy the same identity against the oracle's JVPs.
"""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _state(w, seed=3, noise=0.02):
    f = O.set_state(w)
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(f * (1.0 + noise * rng.normal(size=f.shape)))


SMALL = {
    "extrap": lambda: I.random_smooth(6, 8, seed=3),
    "dirichlet_wall": lambda: I.random_smooth(7, 8, seed=4, bc_kind=(I.BC_DIRICHLET, I.BC_WALL)),
    "wall_extrap": lambda: I.random_smooth(5, 9, seed=5, bc_kind=(I.BC_WALL, I.BC_EXTRAP)),
    "sector_nf1": lambda: I.random_smooth(6, 5, seed=6, n_f=1),
    "smallest": lambda: I.random_smooth(3, 2, seed=7),
    # RM state with its shock and interface, made non-uniform by the noise:
    # where two neighbours are bitwise equal the switch function sits on its
    # kink and the two implementations' roundings pick different branches.
    "rm_noisy": lambda: I.rm(n_r=9, n_theta=6),
}


def _dev(a, dtype):
    return torch.as_tensor(a, dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", list(SMALL))
def test_fp64_adjoint_step_equals_oracle_vjp(name):
    w = SMALL[name]()
    f = _state(w)
    lam = np.random.default_rng(9).normal(size=f.shape)
    want = O.adjoint_step(w, f, lam)
    with P.PCLB(w, precision="fp64") as g:
        got = g.adjoint_step(_dev(f, torch.float64), _dev(lam, torch.float64)).cpu().numpy()
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= 1e-12, err


# Multi-tile grids for entry-by-entry comparison: the adjoint kernels' tiles
# are 32 (r) x 8 (theta) in FP64 and 32 x 16 in FP32, so these span several
# tiles with ragged tails in both directions, the seam rows, both walls of
# every kind and sectors.
MULTI = {
    "dirichlet_wall_67x35": lambda: I.random_smooth(67, 35, seed=41, bc_kind=(I.BC_DIRICHLET, I.BC_WALL)),
    "wall_extrap_sector3_67x35": lambda: I.random_smooth(67, 35, seed=42, n_f=3,
                                                         bc_kind=(I.BC_WALL, I.BC_EXTRAP)),
    "extrap_99x21": lambda: I.random_smooth(99, 21, seed=43),
    "extrap_dirichlet_sector1_70x17": lambda: I.random_smooth(70, 17, seed=44, n_f=1,
                                                              bc_kind=(I.BC_EXTRAP, I.BC_DIRICHLET)),
    "rm_noisy_96x40": lambda: I.rm(n_r=96, n_theta=40),
}


def _all_entries(shape):
    q, t, r = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    return q.ravel(), t.ravel(), r.ravel()


@pytest.mark.parametrize("name", list(MULTI))
def test_fp64_adjoint_equals_oracle_entry_by_entry_on_multi_tile_grids(name):
    """Every entry of lam^n -- tile edges, seam rows, wall columns, ragged
    tails -- against the oracle's entry from forward-mode sweeps over the
    nodes that read it, within 1e-12 of max|lam^n|."""
    w = MULTI[name]()
    f = _state(w, seed=51)
    lam = np.random.default_rng(52).normal(size=f.shape)
    with P.PCLB(w, precision="fp64") as g:
        got = g.adjoint_step(_dev(f, torch.float64), _dev(lam, torch.float64)).cpu().numpy()
        assert g.status_flags() == 0
    q, t, r = _all_entries(f.shape)
    want = O.adjoint_entries(w, f, lam, q, t, r).reshape(f.shape)
    err = np.abs(got - want) / np.max(np.abs(want))
    assert err.max() <= 1e-12, (err.max(), np.unravel_index(np.argmax(err), err.shape))


@pytest.mark.parametrize("name", list(MULTI))
def test_fp32_adjoint_close_to_oracle_entry_by_entry_on_multi_tile_grids(name):
    w = MULTI[name]()
    f = _state(w, seed=53).astype(np.float32).astype(np.float64)
    lam = np.random.default_rng(54).normal(size=f.shape).astype(np.float32).astype(np.float64)
    with P.PCLB(w, precision="fp32") as g:
        got = g.adjoint_step(_dev(f, torch.float32), _dev(lam, torch.float32)).double().cpu().numpy()
    q, t, r = _all_entries(f.shape)
    want = O.adjoint_entries(w, f, lam, q, t, r).reshape(f.shape)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= 1e-4, err


@pytest.mark.parametrize("shape,bc", [((40, 20), (I.BC_EXTRAP, I.BC_EXTRAP)),
                                      ((67, 13), (I.BC_DIRICHLET, I.BC_WALL)),
                                      ((33, 9), (I.BC_WALL, I.BC_DIRICHLET))])
def test_fp64_adjoint_transpose_identity_on_multi_tile_grids(shape, bc):
    w = I.random_smooth(*shape, seed=11, bc_kind=bc)
    f = _state(w)
    rng = np.random.default_rng(12)
    lam = rng.normal(size=f.shape)
    with P.PCLB(w, precision="fp64") as g:
        adj = g.adjoint_step(_dev(f, torch.float64), _dev(lam, torch.float64)).cpu().numpy()
    for _ in range(2):
        df = rng.normal(size=f.shape)
        lhs = np.sum(lam * O.step_jvp(w, f, df))
        rhs = np.sum(adj * df)
        assert rhs == pytest.approx(lhs, rel=1e-11, abs=1e-11 * np.sum(np.abs(lam * df)))


@pytest.mark.parametrize("name", [n for n in SMALL if n != "rm_noisy"])
def test_fp32_adjoint_step_close_to_oracle(name):
    w = SMALL[name]()
    f = _state(w).astype(np.float32).astype(np.float64)
    lam = np.random.default_rng(9).normal(size=f.shape).astype(np.float32).astype(np.float64)
    want = O.adjoint_step(w, f, lam)
    with P.PCLB(w, precision="fp32") as g:
        got = g.adjoint_step(_dev(f, torch.float32), _dev(lam, torch.float32)).double().cpu().numpy()
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= 1e-4, err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_on_saved_states_equals_packed_form(prec):
    w = I.random_smooth(37, 19, seed=13)
    with P.PCLB(w, precision=prec) as g:
        g.set_state().step(2)
        st = g.save_state()
        f = g.get_f()
        lam = torch.randn((33, 19, 37), dtype=g.dtype, device="cuda")
        a = g.adjoint_step(f, lam)
        g.lambda_set(lam).adjoint_state(st)
        b = g.lambda_get()
        assert torch.equal(a, b)
        g.lambda_set(lam).adjoint_state(None)   # the current state is the same one
        assert torch.equal(g.lambda_get(), a)


def test_fp64_field_vjps_are_transposes_of_oracle_jvps():
    w = I.random_smooth(35, 17, seed=14, bc_kind=(I.BC_DIRICHLET, I.BC_EXTRAP))
    rng = np.random.default_rng(15)
    fields = [np.array(x) for x in w.fields()]
    f = _state(w)
    with P.PCLB(w, precision="fp64") as g:
        # moments: <g, J_m df> = <J_m^T g, df>
        gs = [rng.normal(size=fields[0].shape) for _ in range(4)]
        g.set_f(_dev(f, torch.float64)).moments_vjp(*gs)
        lam = g.lambda_get().cpu().numpy()
        df = rng.normal(size=f.shape)
        jv = O.fields_jvp(w, f, df)
        lhs = sum(np.sum(a * b) for a, b in zip(gs, jv))
        assert np.sum(lam * df) == pytest.approx(lhs, rel=1e-11)
        # set_state: <lam, J_s dfields> = <J_s^T lam, dfields>
        lam2 = rng.normal(size=f.shape)
        g.lambda_set(_dev(lam2, torch.float64))
        grads = [x.cpu().numpy() for x in g.set_state_vjp(*fields)]
        dfields = [rng.normal(size=fields[0].shape) for _ in range(4)]
        jv2 = O.set_state_jvp(w, fields, dfields)
        rhs = sum(np.sum(a * b) for a, b in zip(grads, dfields))
        assert rhs == pytest.approx(np.sum(lam2 * jv2), rel=1e-11)
