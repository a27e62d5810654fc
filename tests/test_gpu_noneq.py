"""Parity of the non-equilibrium manifestations (Sec. IV, pclb_noneq) with the
oracle: the moments M_m(f), the departures Delta_m, the central moments
M*_m(f) and the central departures Delta*_m, all 12 polar components.

Errors are measured against the size of the terms each sum adds up, the
absolute moment sum_q |f_q| |c_q|^k of the same order k (k = 2 for M_2, 3 for
M_3 and M_{3,1}, 4 for M_{4,2}; c = v, or v - u for the central groups): a
sum of 33 rounded products is accurate to a few units of rounding of that
size, however much the terms cancel (near equilibrium the central third
moments and all departures are small differences of large terms); the same
for the 65 and 97 products of the larger velocity sets.  FP64:
1e-14 of it.  FP32 (inputs rounded to float, the oracle run on the rounded
values, the equilibrium evaluated in float as the step does): 5e-7.  At
equilibrium the departures vanish to the same rounding on the GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALL = P.NEQ_M | P.NEQ_DELTA | P.NEQ_MSTAR | P.NEQ_DSTAR

CASES = {
    "smooth_ragged": lambda: I.random_smooth(37, 19, seed=1),
    "sector_nf1": lambda: I.random_smooth(35, 17, seed=3, n_f=1),
    "rm": lambda: I.rm(n_r=96, n_theta=64),
    "kh": lambda: I.kh(n_r=64, n_theta=96),
    # the 16- and 24-direction sets of Table I (Q = 65, 97)
    "n16_ragged": lambda: I.random_smooth(37, 19, seed=5, n_dirs=16, n_f=16),
    "n24_sector": lambda: I.random_smooth(33, 12, seed=6, n_dirs=24, n_f=5),
}


ORDER = np.array([2, 2, 2, 3, 3, 3, 3, 3, 3, 4, 4, 4])


def _abs_scale(w, f, central):
    """Per component: max over nodes of sum_q |f_q| |c_q|^k, k its order."""
    vx, vy, _ = O.dvm(w.n_dirs, w.speeds)
    cx = vx[:, None, None]
    cy = vy[:, None, None]
    if central:
        rho, ur, ut, _ = O.fields(w, f)
        th = np.asarray(I.angles(w.n_theta, w.n_dirs, w.n_f))[:, None]
        cx = cx - (ur * np.cos(th) - ut * np.sin(th))[None]
        cy = cy - (ur * np.sin(th) + ut * np.cos(th))[None]
    speed = np.sqrt(cx * cx + cy * cy)
    by_order = {k: np.max(np.sum(np.abs(f) * speed ** k, axis=0)) for k in (2, 3, 4)}
    return np.array([by_order[k] for k in ORDER])


def _noisy(w, seed=21):
    f = O.set_state(w)
    return np.ascontiguousarray(f * (1.0 + 0.03 * np.random.default_rng(seed).normal(size=f.shape)))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 5e-7)])
@pytest.mark.parametrize("name", list(CASES))
def test_noneq_matches_oracle(name, prec, tol):
    w = CASES[name]()
    f = _noisy(w)
    dtype = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        f = f.astype(np.float32).astype(np.float64)
    want = O.noneq(w, f, ALL)
    with P.PCLB(w, precision=prec) as g:
        got = g.set_f(torch.as_tensor(f, dtype=dtype, device="cuda")).noneq(ALL).double().cpu().numpy()
        assert g.status_flags() == 0
    assert got.shape == want.shape == (4, 12, w.n_theta, w.n_r)
    scales = {False: _abs_scale(w, f, False), True: _abs_scale(w, f, True)}
    for grp, label in enumerate(("M", "Delta", "M*", "Delta*")):
        err = np.max(np.abs(got[grp] - want[grp]), axis=(1, 2)) / scales[grp >= 2]
        assert np.max(err) <= tol, (label, err)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-14), ("fp32", 5e-7)])
def test_departures_vanish_at_equilibrium_on_gpu(prec, tol):
    w = I.kh(n_r=64, n_theta=96)
    with P.PCLB(w, precision=prec) as g:
        g.set_state()
        out = g.noneq(ALL).double().cpu().numpy()
        f = g.get_f().double().cpu().numpy()
    for grp, central in ((1, False), (3, True)):
        err = np.max(np.abs(out[grp]), axis=(1, 2)) / _abs_scale(w, f, central)
        assert np.max(err) <= tol, (grp, err)


def test_single_groups_select_the_same_fields():
    w = CASES["smooth_ragged"]()
    f = _noisy(w)
    with P.PCLB(w, precision="fp64") as g:
        g.set_f(torch.as_tensor(f, device="cuda"))
        both = g.noneq(P.NEQ_DELTA | P.NEQ_DSTAR).cpu().numpy()
        d = g.noneq(P.NEQ_DELTA).cpu().numpy()
        ds = g.noneq(P.NEQ_DSTAR).cpu().numpy()
    assert np.array_equal(both[0], d[0]) and np.array_equal(both[1], ds[0])


def test_noneq_errors():
    w = CASES["smooth_ragged"]()
    with P.PCLB(w, precision="fp32") as g:
        with pytest.raises(P.PCLBError) as e:
            g.noneq(P.NEQ_M)
        assert e.value.code == 7   # PCLB_ESTATE
        g.set_state()
        with pytest.raises(P.PCLBError) as e:
            g.noneq(16)
        assert e.value.code == 1   # PCLB_EINVAL
