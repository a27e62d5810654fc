"""The convection schemes and the relaxation variant the paper compares
(pclb_set_scheme: MWB, Warming-Beam, Lax-Wendroff, second-order upwind;
analytic or forward-Euler relaxation) against the oracle: one step from the
same noisy state, FP64 within 1e-12 and FP32 within 2e-6 of max|f|; and the
entry point's refusals."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GRIDS = {
    "smooth_ragged": lambda: I.random_smooth(37, 19, seed=1),
    "dirichlet_wall": lambda: I.random_smooth(40, 24, seed=2, bc_kind=(I.BC_DIRICHLET, I.BC_WALL)),
    "sector_nf1": lambda: I.random_smooth(35, 17, seed=3, n_f=1),
}
VARIANTS = [(s, r) for s in (P.SCHEME_MWB, P.SCHEME_WB, P.SCHEME_LW, P.SCHEME_UPWIND2)
            for r in (P.RELAX_EXACT, P.RELAX_EULER)]


def _noisy(w, seed=11):
    f = O.set_state(w)
    return np.ascontiguousarray(f * (1.0 + 0.01 * np.random.default_rng(seed).normal(size=f.shape)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("scheme,relax", VARIANTS)
@pytest.mark.parametrize("name", list(GRIDS))
def test_variant_one_step_matches_oracle(name, scheme, relax, prec, tol):
    w = GRIDS[name]()
    w.scheme, w.relaxation = scheme, relax
    f0 = _noisy(w)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        f0 = f0.astype(np.float32).astype(np.float64)
    want = O.step(w, f0)
    with P.PCLB(w, precision=prec) as g:
        got = g.set_f(torch.as_tensor(f0, dtype=dtype, device="cuda")).step(1).get_f().double().cpu().numpy()
        assert g.status_flags() == 0
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) <= tol


def test_scheme_can_be_switched_back():
    w = GRIDS["smooth_ragged"]()
    f0 = _noisy(w)
    with P.PCLB(w, precision="fp64") as g:
        a = g.set_f(torch.as_tensor(f0, device="cuda")).step(1).get_f().cpu().numpy()
        g.set_scheme(P.SCHEME_LW, P.RELAX_EULER).set_f(torch.as_tensor(f0, device="cuda")).step(1)
        g.set_scheme(P.SCHEME_MWB, P.RELAX_EXACT)
        b = g.set_f(torch.as_tensor(f0, device="cuda")).step(1).get_f().cpu().numpy()
    assert np.array_equal(a, b)


def test_set_scheme_refusals():
    w = I.random_smooth(20, 12, seed=4, tau=1e-5)   # dt >> tau
    with P.PCLB(w, precision="fp32") as g:
        with pytest.raises(P.PCLBError) as e:
            g.set_scheme(7, 0)
        assert e.value.code == 1        # PCLB_EINVAL
        with pytest.raises(P.PCLBError) as e:
            g.set_scheme(0, P.RELAX_EULER)
        assert e.value.code == 6        # PCLB_ECFL: forward Euler with dt > 2 tau
        g.set_scheme(P.SCHEME_WB, P.RELAX_EXACT).set_state()
        f = g.get_f()
        with pytest.raises(P.PCLBError) as e:
            g.adjoint_step(f, torch.zeros_like(f))
        assert e.value.code == 8        # PCLB_EUNSUPPORTED: the adjoint is MWB only
