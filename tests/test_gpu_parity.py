"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64 path: one step within 1e-12 of max|f| of the oracle, from identical
inputs.  FP32 path: one step within 2e-6 of max|f|; after many steps the
macroscopic fields within relative L2 1e-5 (smooth flows) or relative L1
1e-4 (shocked flows) of the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cases():
    return {
        # sizes chosen to span several tiles (32 x 16 nodes) with ragged tails
        "smooth_ragged": lambda: I.random_smooth(37, 19, seed=1),
        "smooth_dirichlet_wall": lambda: I.random_smooth(40, 24, seed=2, bc_kind=(I.BC_DIRICHLET, I.BC_WALL)),
        "exact_tile": lambda: I.random_smooth(32, 16, seed=5),
        "outer_ghost_in_penultimate_tile": lambda: I.random_smooth(33, 20, seed=6),
        "two_tiles_plus_two": lambda: I.random_smooth(66, 35, seed=7, bc_kind=(I.BC_WALL, I.BC_DIRICHLET)),
        "sector_nf1": lambda: I.random_smooth(35, 17, seed=3, n_f=1),
        "sector_nf3": lambda: I.random_smooth(20, 9, seed=8, n_f=3),
        "smallest": lambda: I.random_smooth(3, 2, seed=4),
        "narrow_theta": lambda: I.random_smooth(50, 3, seed=9),
        "rot": lambda: I.rot(),
        "shock": lambda: I.shock(n_r=300, n_theta=16),
        "rm": lambda: I.rm(n_r=96, n_theta=64),
        "kh": lambda: I.kh(n_r=64, n_theta=96),
    }


CASES = _cases()


def _noisy_state(w, seed=11):
    f = O.set_state(w)
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(f * (1.0 + 0.01 * rng.normal(size=f.shape)))


def _to_dev(a, dtype):
    return torch.as_tensor(a, dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_one_step_matches_oracle(name):
    w = CASES[name]()
    f0 = _noisy_state(w)
    want = O.step(w, f0)
    with P.PCLB(w, precision="fp64") as g:
        g.set_f(_to_dev(f0, torch.float64)).step(1)
        got = g.get_f().cpu().numpy()
        assert g.status_flags() == 0
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= 1e-12, err


@pytest.mark.parametrize("name", ["smooth_ragged", "sector_nf1", "rot", "shock", "rm", "kh"])
def test_fp64_ten_steps_match_oracle(name):
    w = CASES[name]()
    f0 = _noisy_state(w)
    want = O.run(w, f0, 10)
    with P.PCLB(w, precision="fp64") as g:
        got = g.set_f(_to_dev(f0, torch.float64)).step(10).get_f().cpu().numpy()
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= 1e-11, err


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_one_step_matches_oracle(name):
    w = CASES[name]()
    f0 = _noisy_state(w).astype(np.float32).astype(np.float64)
    want = O.step(w, f0)
    with P.PCLB(w, precision="fp32") as g:
        got = g.set_f(_to_dev(f0, torch.float32)).step(1).get_f().cpu().numpy().astype(np.float64)
        assert g.status_flags() == 0
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert err <= 2e-6, err


def _rel(a, b, order):
    a = np.ravel(a)
    b = np.ravel(b)
    return np.linalg.norm(a - b, order) / np.linalg.norm(b, order)


@pytest.mark.parametrize("name,steps,smooth", [
    ("rot", 200, True),
    ("kh", 200, True),
    ("smooth_ragged", 100, True),
    ("shock", 300, False),
    ("rm", 200, False),
])
def test_fp32_many_steps_fields_match_oracle(name, steps, smooth):
    w = CASES[name]()
    f_or = O.run(w, O.set_state(w), steps)
    rho_o, ur_o, ut_o, T_o = O.fields(w, f_or)
    with P.PCLB(w, precision="fp32") as g:
        g.set_state().step(steps)
        rho, ur, ut, T = [x.double().cpu().numpy() for x in g.moments()]
        assert g.status_flags() == 0
    order = 2 if smooth else 1
    tol = 1e-5 if smooth else 1e-4
    u_o = np.stack([ur_o, ut_o])
    u = np.stack([ur, ut])
    errs = (_rel(rho, rho_o, order), _rel(u, u_o, order), _rel(T, T_o, order))
    assert max(errs) <= tol, errs


@pytest.mark.parametrize("prec,tol_f,tol_m", [("fp64", 1e-14, 1e-13), ("fp32", 2e-6, 2e-6)])
def test_set_state_and_moments_match_oracle(prec, tol_f, tol_m):
    w = I.random_smooth(45, 21, seed=12)
    want_f = O.set_state(w)
    with P.PCLB(w, precision=prec) as g:
        got_f = g.set_state().get_f().cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got_f - want_f)) <= tol_f * np.max(np.abs(want_f))
        f_in = want_f * (1 + 0.01 * np.random.default_rng(1).normal(size=want_f.shape))
        g.set_f(_to_dev(f_in, g.dtype))
        got = [x.cpu().numpy().astype(np.float64) for x in g.moments()]
    f_cast = f_in.astype(np.float32).astype(np.float64) if prec == "fp32" else f_in
    want = O.fields(w, f_cast)
    for a, b, name in zip(got, want, ("rho", "u_r", "u_theta", "T")):
        scale = max(np.max(np.abs(b)), 1e-3)
        assert np.max(np.abs(a - b)) <= tol_m * scale, name


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_diagnostics_match_oracle(prec):
    w = I.random_smooth(40, 24, seed=13)
    f = O.set_state(w)
    if prec == "fp32":   # the oracle sees exactly the values the FP32 state holds
        f = f.astype(np.float32).astype(np.float64)
    want = O.diagnostics(w, f)
    with P.PCLB(w, precision=prec) as g:
        got = g.set_f(_to_dev(f, g.dtype)).diagnostics()
    # FP32 moments sum each shell in single precision (relative error ~1e-7 of
    # the shell totals); momentum totals are small differences of large terms,
    # so they get an absolute tolerance scaled by the mass.
    tol = 1e-13 if prec == "fp64" else 2e-7
    assert got[:6] == pytest.approx(want, rel=tol, abs=tol * want[0])
    assert got[6] == w.n_r * w.n_theta


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_get_set_f_round_trip_is_bitwise(prec):
    w = I.random_smooth(35, 18, seed=14)
    with P.PCLB(w, precision=prec) as g:
        f = _to_dev(_noisy_state(w), g.dtype)
        back = g.set_f(f).get_f()
        assert torch.equal(back, f)
        # the state survives a step and restore bitwise
        g.step(3)
        s = g.get_f()
        g.step(2)
        g.set_f(s)
        assert torch.equal(g.get_f(), s)


def test_nonphysical_input_sets_status_flag():
    w = I.random_smooth(20, 10, seed=15)
    with P.PCLB(w, precision="fp32") as g:
        rho = w.rho.copy()
        rho[3, 4] = -1.0
        g.set_state(rho=rho)
        assert g.status_flags(clear=True) & P.FLAG_NONPHYS
        assert g.status_flags() == 0
        g.set_state()
        g.step(2)
        assert g.status_flags() == 0


def test_step_before_state_is_refused():
    w = I.random_smooth(20, 10, seed=16)
    with P.PCLB(w, precision="fp32") as g:
        with pytest.raises(P.PCLBError) as e:
            g.step(1)
        assert e.value.code == 7


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("pinned_in,pinned_out", [(True, False), (False, False), (True, True)])
def test_run_host_equals_device_path(prec, pinned_in, pinned_out):
    """pclb_run_host gives the device path's fields bit for bit, whether the
    kernels access page-locked buffers directly (all pinned) or the fields are
    staged through the workspace (any pageable buffer)."""
    w = I.random_smooth(50, 30, seed=17)
    dtype = torch.float32 if prec == "fp32" else torch.float64
    with P.PCLB(w, precision=prec) as g:
        dev = [x.cpu() for x in g.set_state().step(4).moments()]
        ins = [torch.as_tensor(x, dtype=dtype) for x in w.fields()]
        ins = [x.pin_memory() if pinned_in else x for x in ins]
        outs = [torch.full((w.n_theta, w.n_r), float("nan"), dtype=dtype) for _ in range(4)]
        outs = [x.pin_memory() if pinned_out else x for x in outs]
        host = g.run_host(*ins, 4, outs)
    for a, b in zip(host, dev):
        assert torch.equal(a, b)
