"""Temperature recovery and the step at high Mach number (GPU).

T = (e - rho u^2 / 2) / rho (Eqs. 3-5) cancels when u^2 / 2E >> 1.  The FP64
path sums the moments and recovers T in FP64.  The FP32 path sums each shell
in FP32, combines the shell totals and recovers T in float-float: its T
differs from the oracle's T of the same FP32 values by at most ~2 (u^2/2E)
units in the last place of FP32.  That is the size by which T already moves
when each stored FP32 value of f moves by its rounding (the conditioning of T
with respect to f is u^2/2E), so recovering T in FP64 from exact sums would
not make the FP32 state's temperature more accurate by more than a small
factor at any Mach number; it would take exact sums of 33 values per node at
GB300's FP64 rate.  Checked here on distributions whose sums are exact in
FP32 (dyadic values: a beam along one direction of shells 3 and 4 with a
small spread) at u^2/2E from ~60 to ~2400, where the plain FP32 formula
would be off by more than the bound.

At such Mach numbers the octagon's equilibrium itself is the limit: its
values reach (v_max |u| / E)^4 / 24 times rho, so storing f in FP32 loses rho,
u and T whatever the recovery; the FP64 path follows the oracle there to the
equilibrium's own conditioning.
"""
import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I
from paper_1302_7104_gb300 import pclb as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

Q = 33


def _beams(n_r, n_t, seed=4):
    """Dyadic distributions: a beam along direction i of shells 4 and 3,
    weights 1 - eps and eps (eps = 2^-3 .. 2^-9), plus a few small dyadic
    values on other labels; every sum of them is exact in FP32."""
    rng = np.random.default_rng(seed)
    f = np.zeros((Q, n_t, n_r))
    for t in range(n_t):
        for r in range(n_r):
            i = rng.integers(0, 8)
            eps = 2.0 ** -int(rng.integers(3, 10))
            f[1 + 3 * 8 + i, t, r] = 1.0 - eps
            f[1 + 2 * 8 + i, t, r] = eps
            for q in rng.integers(0, Q, 4):
                f[q, t, r] += int(rng.integers(1, 8)) * 2.0 ** -14
    assert np.array_equal(f.astype(np.float32).astype(np.float64), f)
    return f


def _cancelling_T_in_fp32(w, f):
    """T = (e - |j|^2 / 2 rho) / rho with every sum and product in FP32, for
    comparison: the formula the recovery avoids."""
    vx, vy, _ = O.dvm(8, I.SPEEDS)                            # Cartesian velocities of the labels
    f32 = f.astype(np.float32)
    vx, vy = vx.astype(np.float32), vy.astype(np.float32)
    rho = f32.sum(axis=0, dtype=np.float32)
    jx = np.tensordot(vx, f32, axes=(0, 0)).astype(np.float32)
    jy = np.tensordot(vy, f32, axes=(0, 0)).astype(np.float32)
    e = np.tensordot((np.float32(0.5) * (vx * vx + vy * vy)).astype(np.float32), f32, axes=(0, 0)).astype(np.float32)
    return ((e - np.float32(0.5) * (jx * jx + jy * jy) / rho) / rho).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_temperature_recovery_at_high_mach(prec):
    n_r, n_t = 40, 24
    w = I.uniform(n_r, n_t, rho=1.0, ux=0.0, uy=0.0, T=1.0, cfl=I.STABLE_CFL)
    f = _beams(n_r, n_t)
    rho, ur, ut, T = O.fields(w, f)
    mach2 = (ur ** 2 + ut ** 2) / (2.0 * T)
    assert mach2.min() > 50.0 and mach2.max() > 2000.0
    dtype = torch.float32 if prec == "fp32" else torch.float64
    with P.PCLB(w, precision=prec) as g:
        g.set_f(torch.as_tensor(f, dtype=dtype, device="cuda"))
        got = [x.double().cpu().numpy() for x in g.moments()]
    err = np.abs(got[3] - T) / T
    # within (4 u^2/2E + 4) units in the last place node by node (measured:
    # 1.9 u^2/2E at most in FP32; FP64 sums are exact here, its recovery
    # still rounds at the same conditioning: 2.5 u^2/2E at most)
    tol = (4.0 * mach2 + 4.0) * (2.0 ** -24 if prec == "fp32" else 2.0 ** -52)
    print(prec, "high-Mach T recovery: max relative error", err.max(), "max error / (u^2/2E ulp)",
          np.max(err / (mach2 * 2.0 ** -24)), "at u^2/2E up to", mach2.max())
    assert np.all(err <= tol), np.max(err / tol)
    assert np.max(np.abs(got[0] - rho)) <= (2 ** -24 if prec == "fp32" else 1e-15)
    if prec == "fp32":
        plain = np.abs(_cancelling_T_in_fp32(w, f) - T) / T
        assert np.any(plain > tol)             # the same formula with FP32 products and sums exceeds it


def test_fp64_step_matches_oracle_at_mach_5():
    """Uniform flow at Mach 5 (|u| = 1, T = 0.02: u^2/2E = 25) with a small
    non-equilibrium part: the equilibrium's values reach ~6e4 rho and its
    polynomial (x = v.u/E up to 224) cancels by ~1e8, so even two FP64
    evaluations in different orders differ at ~1e-8 of max|f| (measured
    3.5e-8 between the FP64 path and the oracle): the FP64 path follows the
    oracle to that conditioning, where an FP32 state keeps nothing (its
    rounding of max|f| alone is ~4e-3 rho)."""
    w = I.uniform(40, 24, rho=1.0, ux=1.0, uy=0.0, T=0.02, cfl=I.STABLE_CFL, tau=1e-3)
    f = O.set_state(w)
    f = f * (1.0 + 1e-9 * np.random.default_rng(5).normal(size=f.shape))
    want = O.step(w, f)
    with P.PCLB(w, precision="fp64") as g:
        got = g.set_f(torch.as_tensor(f, device="cuda")).step(1).get_f().cpu().numpy()
        assert g.status_flags() == 0
    assert np.max(np.abs(f)) > 1e4
    assert np.max(np.abs(got - want)) <= 1e-7 * np.max(np.abs(want))
