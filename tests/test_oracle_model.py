"""Pins of the oracle's velocity model, weights, equilibrium and moments
against facts the paper and the mathematics fix (no GPU)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1302_7104_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table1_coefficients.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, ni, b0, b4, b3, b2, b1 = line.split()
        rows[int(ni)] = (float(b0), float(b1), float(b2), float(b3), float(b4))
    return rows


def test_table1_rows_are_the_closed_form():
    # Table I: B0 = N_i, B4 = 384/N_i, B3 = -48/N_i, B2 = 8/N_i, B1 = -2/N_i.
    for ni, (b0, b1, b2, b3, b4) in _table1().items():
        assert b0 == ni
        assert b4 == pytest.approx(384.0 / ni, rel=1e-15)
        assert b3 == pytest.approx(-48.0 / ni, rel=1e-15)
        assert b2 == pytest.approx(8.0 / ni, rel=1e-15)
        assert b1 == pytest.approx(-2.0 / ni, rel=1e-15)
        assert I.TABLE1_B[ni] == pytest.approx((b0, b1, b2, b3, b4), rel=1e-15)


@pytest.mark.parametrize("n_dirs", [8, 16, 24])
def test_dvm_eq2(n_dirs):
    vx, vy, shell = O.dvm(n_dirs)
    Q = 1 + 4 * n_dirs
    assert len(vx) == Q and shell[0] == 0 and vx[0] == 0 and vy[0] == 0
    for q in range(1, Q):
        k, i = 1 + (q - 1) // n_dirs, 1 + (q - 1) % n_dirs
        assert shell[q] == k
        assert math.hypot(vx[q], vy[q]) == pytest.approx(I.SPEEDS[k], rel=1e-15)
        phi = math.atan2(vy[q], vx[q]) % (2 * math.pi)
        assert phi == pytest.approx(2 * math.pi * (i - 1) / n_dirs, abs=1e-12)


@pytest.mark.parametrize("n_dirs", [8, 16, 24])
@pytest.mark.parametrize("E", [0.2, 0.7, 1.0, 2.5])
def test_weights_match_2d_maxwellian_speed_moments(n_dirs, E):
    # Eqs. (11a)-(11b) make the discrete weights reproduce the speed moments of
    # a 2-D Maxwellian with E = T: sum_q w_q |v_q|^{2n} = 2^n n! E^n, n = 0..4.
    vx, vy, shell = O.dvm(n_dirs)
    F = O.weights(E, n_dirs, I.SPEEDS, I.TABLE1_B[n_dirs])
    w = F[shell]
    v2 = vx * vx + vy * vy
    for n in range(5):
        got = float(np.sum(w * v2 ** n))
        assert got == pytest.approx(2 ** n * math.factorial(n) * E ** n, rel=1e-12), n


def _feq_moment_cases(n):
    rng = np.random.default_rng(1234)
    for _ in range(n):
        yield (rng.uniform(0.1, 3.0), *rng.uniform(-0.7, 0.7, 2), rng.uniform(0.2, 3.0))


@pytest.mark.parametrize("n_dirs", [8, 16])
def test_equilibrium_moment_relations_eqs_3_to_9(n_dirs):
    """Eqs. (3)-(8) as printed; Eq. (9) in its corrected form
    1/2 sum f^eq |v|^2 v v = rho[(2E + u^2/2) E I + (3E + u^2/2) u u]
    (the form the appendix's energy-flux error term uses)."""
    vx, vy, _ = O.dvm(n_dirs)
    V = np.stack([vx, vy], axis=1)
    I2 = np.eye(2)
    for rho, ux, uy, E in _feq_moment_cases(12):
        f = O.feq(rho, ux, uy, E, n_dirs, I.SPEEDS, I.TABLE1_B[n_dirs])
        u = np.array([ux, uy])
        u2 = u @ u
        scale = rho * (1 + E + u2) ** 3

        def close(a, b):
            assert np.max(np.abs(np.asarray(a) - np.asarray(b))) <= 1e-13 * scale

        close(f.sum(), rho)                                          # Eq. (3)
        close(f @ V, rho * u)                                        # Eq. (4)
        c = V - u
        close(0.5 * np.sum(f * np.sum(c * c, axis=1)), rho * E)     # Eq. (5)
        M2 = np.einsum("q,qa,qb->ab", f, V, V)
        close(M2, rho * (E * I2 + np.outer(u, u)))                   # Eq. (6)
        M3 = np.einsum("q,qa,qb,qc->abc", f, V, V, V)
        want3 = rho * (E * (np.einsum("a,bc->abc", u, I2) + np.einsum("b,ac->abc", u, I2)
                            + np.einsum("c,ab->abc", u, I2)) + np.einsum("a,b,c->abc", u, u, u))
        close(M3, want3)                                             # Eq. (7)
        v2 = np.sum(V * V, axis=1)
        close(0.5 * (f * v2) @ V, rho * u * (2 * E + 0.5 * u2))      # Eq. (8)
        M42 = 0.5 * np.einsum("q,qa,qb->ab", f * v2, V, V)
        close(M42, rho * ((2 * E + 0.5 * u2) * E * I2 + (3 * E + 0.5 * u2) * np.outer(u, u)))


def test_eq9_as_printed_fails_for_moving_gas():
    # Documents the reading above: the printed right-hand side of Eq. (9),
    # rho (2E + u^2/2)(E I + u u), misses E u u unless u = 0.
    vx, vy, _ = O.dvm(8)
    V = np.stack([vx, vy], axis=1)
    rho, ux, uy, E = 1.0, 0.5, 0.0, 1.0
    f = O.feq(rho, ux, uy, E, 8, I.SPEEDS, I.TABLE1_B[8])
    u = np.array([ux, uy])
    v2 = np.sum(V * V, axis=1)
    M42 = 0.5 * np.einsum("q,qa,qb->ab", f * v2, V, V)
    printed = rho * (2 * E + 0.125) * (E * np.eye(2) + np.outer(u, u))
    assert abs(M42[0, 0] - printed[0, 0]) == pytest.approx(rho * E * ux * ux, rel=1e-12)


def test_moments_invert_equilibrium():
    for rho, ux, uy, E in _feq_moment_cases(20):
        f = O.feq(rho, ux, uy, E, 8, I.SPEEDS, I.TABLE1_B[8])
        m = O.moments(f, 8, I.SPEEDS)
        assert m == pytest.approx([rho, ux, uy, E], rel=1e-12, abs=1e-13)


def test_moments_of_a_general_distribution():
    # Eqs. (3)-(5) on a non-equilibrium f: rho E = sum f |v|^2/2 - rho u^2/2.
    rng = np.random.default_rng(7)
    vx, vy, _ = O.dvm(8)
    f = rng.uniform(0.01, 0.1, 33)
    rho, ux, uy, E = O.moments(f, 8, I.SPEEDS)
    assert rho == pytest.approx(f.sum(), rel=1e-15)
    assert rho * ux == pytest.approx(f @ vx, rel=1e-14)
    assert rho * uy == pytest.approx(f @ vy, rel=1e-14)
    e_tot = 0.5 * f @ (vx * vx + vy * vy)
    assert rho * E == pytest.approx(e_tot - 0.5 * rho * (ux * ux + uy * uy), rel=1e-13)


def test_equilibrium_is_rotation_covariant():
    # Rotating u by 2 pi / N_i permutes f^eq by one direction within each shell.
    n = 8
    rho, ux, uy, E = 1.2, 0.4, -0.1, 0.9
    a = 2 * math.pi / n
    f0 = O.feq(rho, ux, uy, E, n, I.SPEEDS, I.TABLE1_B[n])
    f1 = O.feq(rho, ux * math.cos(a) - uy * math.sin(a), ux * math.sin(a) + uy * math.cos(a), E, n,
               I.SPEEDS, I.TABLE1_B[n])
    for k in range(1, 5):
        s = slice(1 + (k - 1) * n, 1 + k * n)
        assert np.allclose(np.roll(f0[s], 1), f1[s], rtol=1e-13, atol=1e-15)
    assert f0[0] == pytest.approx(f1[0], rel=1e-14)


def test_hugoniot_helper_reproduces_printed_states():
    path = os.path.join(GOLDEN, "hugoniot_states.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        label, D, rho_h, u_h, p_h = line.split()
        got = I.hugoniot_from_speed(1.0, 0.0, 1.0, float(D))
        assert got == pytest.approx((float(rho_h), float(u_h), float(p_h)), rel=2e-5, abs=2e-6), label
        # and the three relations of Eq. (45) themselves (E = P / rho for gamma = 2)
        r, u, p = got
        Dv = float(D)
        assert r * (u - Dv) == pytest.approx(1.0 * (0.0 - Dv), rel=1e-14)
        assert p - 1.0 == pytest.approx(1.0 * (Dv - 0.0) * (u - 0.0), rel=1e-14)
        assert p / r - 1.0 == pytest.approx(0.5 * (p + 1.0) * (1.0 - 1.0 / r), rel=1e-13)


def test_rm_post_shock_state():
    # Mach 2 inward into (1, 0, P=1): (rho, u_r, P) = (2, -sqrt 2, 5), D = -2 sqrt 2.
    r, u, p, D = I.hugoniot_from_mach(1.0, 0.0, 1.0, 2.0, direction=-1.0)
    assert (r, u, p, D) == pytest.approx((2.0, -math.sqrt(2), 5.0, -2 * math.sqrt(2)), rel=1e-14)
