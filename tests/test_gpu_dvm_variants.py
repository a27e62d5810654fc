"""The larger velocity sets of Table I, N_i = 16 and 24 directions per shell
(Q = 65, 97), on the GPU through the C ABI against the FP64 oracle, with the
bars of the N_i = 8 parity tests: one step within 1e-12 (FP64) or 2e-6 (FP32)
of max|f| from the same noisy state, ten FP64 steps within 1e-11; for full
circles and sectors (label rotation by n_f), every boundary kind including
non-equilibrium ghosts, and every convection scheme and relaxation variant.
Also set_state / moments / get_f against the oracle's equilibrium and
fields, the global integrals, and the reverse-mode and diagnostic entry
points that implement N_i = 8 only refusing."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    # ragged sizes; full circles (n_f = n_dirs) and sectors (n_f < n_dirs)
    "n16_circle": lambda: I.random_smooth(37, 19, seed=21, n_dirs=16, n_f=16),
    "n24_circle": lambda: I.random_smooth(35, 17, seed=22, n_dirs=24, n_f=24),
    "n16_sector_walls": lambda: I.random_smooth(40, 24, seed=23, n_dirs=16, n_f=4,
                                                bc_kind=(I.BC_DIRICHLET, I.BC_WALL)),
    "n24_sector_nf5": lambda: I.random_smooth(20, 9, seed=24, n_dirs=24, n_f=5),
    "n16_neq_ghosts": lambda: I.random_smooth(33, 12, seed=25, n_dirs=16, n_f=16,
                                              bc_kind=(I.BC_EXTRAP | I.BC_NEQ, I.BC_WALL | I.BC_NEQ)),
    "n24_smallest": lambda: I.random_smooth(3, 2, seed=26, n_dirs=24, n_f=24),
}


def _noisy(w, seed=11):
    f = O.set_state(w)
    return np.ascontiguousarray(f * (1.0 + 0.01 * np.random.default_rng(seed).normal(size=f.shape)))


def _dev(a, dtype):
    return torch.as_tensor(a, dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_one_step_matches_oracle(name):
    w = CASES[name]()
    assert w.q == 1 + 4 * w.n_dirs
    f0 = _noisy(w)
    want = O.step(w, f0)
    with P.PCLB(w, precision="fp64") as g:
        got = g.set_f(_dev(f0, torch.float64)).step(1).get_f().cpu().numpy()
        assert g.status_flags() == 0
    assert got.shape == (w.q, w.n_theta, w.n_r)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-12


@pytest.mark.parametrize("name", ["n16_circle", "n24_sector_nf5", "n16_neq_ghosts"])
def test_fp64_ten_steps_match_oracle(name):
    w = CASES[name]()
    f0 = _noisy(w)
    want = O.run(w, f0, 10)
    with P.PCLB(w, precision="fp64") as g:
        got = g.set_f(_dev(f0, torch.float64)).step(10).get_f().cpu().numpy()
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 1e-11


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_one_step_matches_oracle(name):
    w = CASES[name]()
    f0 = _noisy(w).astype(np.float32).astype(np.float64)
    want = O.step(w, f0)
    with P.PCLB(w, precision="fp32") as g:
        got = g.set_f(_dev(f0, torch.float32)).step(1).get_f().double().cpu().numpy()
        assert g.status_flags() == 0
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= 2e-6


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("scheme,relax", [(s, r) for s in (P.SCHEME_MWB, P.SCHEME_WB, P.SCHEME_LW, P.SCHEME_UPWIND2)
                                          for r in (P.RELAX_EXACT, P.RELAX_EULER)])
def test_schemes_one_step_match_oracle(scheme, relax, prec, tol):
    w = CASES["n16_sector_walls"]()
    w.scheme, w.relaxation = scheme, relax
    dtype = torch.float64 if prec == "fp64" else torch.float32
    f0 = _noisy(w)
    if prec == "fp32":
        f0 = f0.astype(np.float32).astype(np.float64)
    want = O.step(w, f0)
    with P.PCLB(w, precision=prec) as g:
        got = g.set_f(_dev(f0, dtype)).step(1).get_f().double().cpu().numpy()
        assert g.status_flags() == 0
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= tol


@pytest.mark.parametrize("name", ["n16_circle", "n24_circle"])
def test_set_state_and_moments_match_oracle(name):
    w = CASES[name]()
    want_f = O.set_state(w)
    with P.PCLB(w, precision="fp64") as g:
        g.set_state()
        f = g.get_f().cpu().numpy()
        assert np.max(np.abs(f - want_f)) / np.max(np.abs(want_f)) <= 1e-13
        g.set_f(_dev(_noisy(w), torch.float64))
        got = [x.cpu().numpy() for x in g.moments()]
        want = O.fields(w, _noisy(w))
        for a, b in zip(got, want):
            assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))
        d = g.diagnostics()
        want_d = O.diagnostics(w, _noisy(w))
        assert np.allclose(d[:6], want_d, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n_dirs", [16, 24])
def test_uniform_state_stays_uniform_and_conserves(n_dirs):
    w = I.uniform(24, 16, n_dirs=n_dirs, n_f=n_dirs)
    with P.PCLB(w, precision="fp64") as g:
        g.set_state()
        d0 = g.diagnostics()
        f0 = g.get_f().cpu().numpy()
        f1 = g.step(5).get_f().cpu().numpy()
        d1 = g.diagnostics()
    assert np.max(np.abs(f1 - f0)) <= 1e-13 * np.max(np.abs(f0))
    assert np.allclose(d1[:4], d0[:4], rtol=1e-13, atol=1e-15)


def test_reverse_mode_refuses_larger_sets():
    w = CASES["n16_circle"]()
    with P.PCLB(w, precision="fp64") as g:
        g.set_state()
        rho = g.moments()[0]
        with pytest.raises(P.PCLBError) as e:
            g.moments_vjp(torch.ones_like(rho))
        assert e.value.code == 8                      # PCLB_EUNSUPPORTED


@pytest.mark.parametrize("n_dirs", [16, 24])
def test_fp32_many_steps_track_fp64(n_dirs):
    """The FP32 generic step (moments from float shell sums combined in
    double) over 200 steps against the FP64 generic step (itself within 1e-12
    per step of the oracle): relative L2 of rho, u and T within 1e-5."""
    w = I.random_smooth(200, 96, seed=27, n_dirs=n_dirs, n_f=n_dirs)

    def fields(prec):
        with P.PCLB(w, precision=prec) as g:
            g.set_state().step(200)
            assert g.status_flags() == 0
            out = [x.double() for x in g.moments()]
            g.sync()
            return out

    rho, ur, ut, T = fields("fp32")
    rho_d, ur_d, ut_d, T_d = fields("fp64")

    def rel(x, y):
        return (torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y)).item()

    errs = {"rho": rel(rho, rho_d), "u": rel(torch.stack([ur, ut]), torch.stack([ur_d, ut_d])), "T": rel(T, T_d)}
    print(n_dirs, "200 steps, FP32 vs FP64:", errs)
    assert max(errs.values()) <= 1e-5, errs
