"""Pins of the AT coefficients (Eq. 14-15, Table 1) and of the Runge-Kutta tables
(Eq. 10, Table 2; Carpenter-Kennedy RK4(5))."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from conftest import golden


def test_at_table1_exact():
    for row in golden("at_coeffs_table1.txt"):
        order, k = int(row[0]), int(row[1])
        ref = np.array([float(v) for v in row[2:2 + order]])
        c = O.at_coeffs(order - 1, float(k))
        np.testing.assert_allclose(c, ref, rtol=0, atol=1e-11)


def lagrange_extrapolation_weights(np_, km):
    # independent closed form: extrapolate to 0 from nodes -(km+l), l = 0..np_
    # weight_l = prod_{j != l} (km + j) / (j - l), evaluated with exact rationals
    km = Fraction(km).limit_denominator(10 ** 12)
    w = []
    for l in range(np_ + 1):
        v = Fraction(1)
        for j in range(np_ + 1):
            if j != l:
                v *= (km + j) / Fraction(j - l)
        w.append(float(v))
    return np.array(w)


@pytest.mark.parametrize("np_", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("km", [0.0, 0.5, 1.0, 1.3772, 2.0, 3.75, 4.0])
def test_at_coeffs_equal_lagrange_extrapolation(np_, km):
    c = O.at_coeffs(np_, km)
    ref = lagrange_extrapolation_weights(np_, km)
    scale = max(1.0, np.abs(ref).max())
    np.testing.assert_allclose(c, ref, rtol=0, atol=1e-11 * scale)


@pytest.mark.parametrize("np_", [1, 2, 3, 4])
def test_at_extrapolation_exact_for_polynomials_in_time(np_):
    # the AT combination of values at t = -(km+l) dt reproduces g(0) for deg g <= N_p
    rng = np.random.default_rng(100 + np_)
    for km in (0.0, 1.0, 2.632124764, 3.5):
        c = O.at_coeffs(np_, km)
        g = rng.standard_normal(np_ + 1)
        vals = np.array([np.polyval(g, -(km + l)) for l in range(np_ + 1)])
        assert abs(np.dot(c, vals) - np.polyval(g, 0.0)) < 1e-9 * (1 + abs(g).sum())
        # degree N_p+1 is not reproduced unless t = 0 is itself a stored level (k_m = 0)
        if km == 0.0:
            continue
        g2 = np.concatenate([[1.0], np.zeros(np_ + 1)])
        vals2 = np.array([np.polyval(g2, -(km + l)) for l in range(np_ + 1)])
        assert abs(np.dot(c, vals2)) > 1e-6


def test_lserk_table2_coefficients():
    rows = golden("lserk_table2.txt")
    for scheme, key in (("LSERK22", "rk22"), ("LSERK33", "rk33")):
        a, b, c, _, _ = O.rk_tableau(key)
        mine = [r for r in rows if r[0] == scheme]
        for r in mine:
            m = int(r[1]) - 1
            if r[2] != "-":
                assert a[m] == float(r[2])
            assert b[m] == float(r[3])
            # c_m is derived from a, b (stage m sees w^n + dt sum_j A_mj k_j); the printed
            # value of LSERK(3,3) stage 3 (0.632125000) is b_1 + a_2 = 0.632124764 rounded
            assert abs(c[m] - float(r[4])) < 3e-7


def order_conditions(A, b):
    c = A.sum(axis=1)
    return {
        1: b.sum() - 1.0,
        2: b @ c - 0.5,
        3: (b @ c ** 2 - 1.0 / 3.0, b @ A @ c - 1.0 / 6.0),
        4: (b @ c ** 3 - 0.25, b @ (c * (A @ c)) - 1.0 / 8.0, b @ A @ c ** 2 - 1.0 / 12.0,
            b @ A @ A @ c - 1.0 / 24.0),
    }


def test_rk22_is_second_order():
    _, _, _, A, b = O.rk_tableau("rk22")
    oc = order_conditions(A, b)
    assert abs(oc[1]) < 1e-15 and abs(oc[2]) < 1e-15
    assert max(abs(v) for v in oc[3]) > 1e-3


def test_rk33_is_third_order_to_table_precision():
    _, _, _, A, b = O.rk_tableau("rk33")
    oc = order_conditions(A, b)
    assert abs(oc[1]) < 1e-9 and abs(oc[2]) < 1e-9
    assert max(abs(v) for v in oc[3]) < 1e-9
    assert max(abs(v) for v in oc[4]) > 1e-3


def test_ck45_is_fourth_order():
    _, _, c, A, b = O.rk_tableau("ck45")
    oc = order_conditions(A, b)
    assert abs(oc[1]) < 1e-15 and abs(oc[2]) < 1e-15
    assert max(abs(v) for v in oc[3]) < 1e-15
    assert max(abs(v) for v in oc[4]) < 1e-15
    assert np.all(np.diff(c) > 0) and c[0] == 0.0


@pytest.mark.parametrize("key,order", [("rk22", 2), ("rk33", 3), ("ck45", 4)])
def test_low_storage_recursion_converges_on_linear_ode(key, order):
    # y' = -y, y(0)=1 integrated to t=1 with the low-storage recursion itself
    a, b, c, _, _ = O.rk_tableau(key)
    errs = []
    for nsteps in (10, 20, 40):
        dt = 1.0 / nsteps
        y = 1.0
        for _ in range(nsteps):
            if key == "ck45":
                q = 0.0
                for m in range(len(b)):
                    q = a[m] * q + dt * (-y)
                    y = y + b[m] * q
            else:
                r = y
                for m in range(len(b)):
                    k = -r
                    if m + 1 < len(b):
                        r = y + dt * a[m] * k
                    y = y + dt * b[m] * k
        errs.append(abs(y - math.exp(-1.0)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.15), rates
