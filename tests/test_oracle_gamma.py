"""Pins of the oracle's incomplete gamma Phi_a(t) = t^{-a} Gamma(a,t) = E_{1-a}(t).

Phi enters every term of the splitting of Z (real space a = nu/2, reciprocal
a = (d-nu)/2, near-part Taylor coefficients a + n).  The oracle evaluates it by
quadrature of the defining integral int_1^inf s^{a-1} e^{-ts} ds alone; the pins
are independent of that: scipy's E_n and E_1, adaptive quadrature of the same
integral by QUADPACK, mpmath's generalized exponential integral at 30 digits, the
derivative identity Phi_a' = -Phi_{a+1} and the order recurrence
t Phi_{a+1} = a Phi_a + e^{-t} (integration by parts), which the oracle never uses.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

A_GRID = [x / 2 for x in range(-12, 14)]
T_GRID = [1e-7, 1e-3, 0.05, 0.4, 0.99, 1.0, 1.01, 1.7, 3.0, 7.5, 15.0, 35.0, 80.0]


@pytest.mark.parametrize("a", [a for a in A_GRID if float(a).is_integer() or a > 0])
def test_phi_vs_scipy(oracle_mod, a):
    # a > 0: Gamma(a) Q(a, t) t^{-a}; integer a <= 1: Phi_a = E_{1-a} (scipy expn)
    for t in T_GRID:
        if a > 0:
            ref = special.gamma(a) * special.gammaincc(a, t) * t ** (-a)
        elif a == 1:
            ref = math.exp(-t) / t
        else:
            ref = special.expn(int(1 - a), t)
        got = oracle_mod.phi(a, t)
        assert got == pytest.approx(ref, rel=2e-14), (a, t)


@pytest.mark.parametrize("a", A_GRID)
def test_phi_vs_mpmath_expint(oracle_mod, a):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for t in T_GRID:
        ref = float(mp.expint(1 - a, t))
        assert oracle_mod.phi(a, t) == pytest.approx(ref, rel=1e-14), (a, t)


@pytest.mark.parametrize("a", [-5.5, -2.5, -1.0, -0.5, 0.0, 0.5, 2.0, 4.5])
def test_phi_vs_defining_integral(oracle_mod, a):
    for t in [0.2, 1.3, 6.0]:
        val, err = integrate.quad(lambda s: s ** (a - 1) * math.exp(-t * s), 1.0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
        assert oracle_mod.phi(a, t) == pytest.approx(val, rel=1e-11), (a, t)


def test_e1_vs_scipy(oracle_mod):
    for t in [1e-9, 1e-4, 0.3, 0.999, 1.0, 1.001, 2.5, 10.0, 50.0, 300.0]:
        assert oracle_mod.e1(t) == pytest.approx(special.exp1(t), rel=3e-15)


@pytest.mark.parametrize("a", [-4.5, -3.0, -1.5, -0.5, 0.0, 0.5, 1.5, 3.0])
def test_phi_derivative_identity(oracle_mod, a):
    # Phi_a'(t) = -Phi_{a+1}(t), checked by a 4th-order central difference
    for t in [0.7, 2.2, 5.0]:
        h = 1e-3 * t
        f = lambda x: oracle_mod.phi(a, x)
        d = (-f(t + 2 * h) + 8 * f(t + h) - 8 * f(t - h) + f(t - 2 * h)) / (12 * h)
        assert d == pytest.approx(-oracle_mod.phi(a + 1, t), rel=1e-9)


@pytest.mark.parametrize("a", [-5.5, -3.0, -0.5])
def test_phi_at_zero(oracle_mod, a):
    assert oracle_mod.phi(a, 0.0) == pytest.approx(-1.0 / a, rel=1e-15)
    # small t: Phi_a(t) = Gamma(a) t^{-a} - 1/a + O(t)
    t = 1e-12
    sing = 0.0 if float(a).is_integer() else special.gamma(a) * t ** (-a)  # log case: t^m log t
    assert oracle_mod.phi(a, t) == pytest.approx(sing - 1.0 / a, abs=1e-11)


@pytest.mark.parametrize("a", [-5.3, -2.05, -0.7, -0.1, 0.05, 0.3, 1.15, 2.8, 6.45])
def test_phi_general_order(oracle_mod, a):
    # orders of non-integer exponents (a = nu/2, (d - nu)/2 for real nu): mpmath at 30 digits,
    # and scipy's regularised upper incomplete gamma for a > 0
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for t in [1e-9, 1e-4, 0.05, 0.49, 0.5, 0.99, 1.0, 2.7, 11.0, 40.0, 150.0]:
        ref = float(mp.expint(1 - a, t))
        assert oracle_mod.phi(a, t) == pytest.approx(ref, rel=3e-15), (a, t)
        if a > 0:
            assert oracle_mod.phi(a, t) == pytest.approx(special.gamma(a) * special.gammaincc(a, t) * t ** (-a),
                                                         rel=1e-13), (a, t)


def test_phi_vs_mpmath_dense_grid(oracle_mod):
    # every order the oracle needs (reciprocal a down to -11/2, Taylor orders a + n up to
    # a + 2 ell), t from the h = 0 term near k = 0 to beyond every cutoff
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    worst = 0.0
    for a in [x / 2 for x in range(-13, 29)]:
        for t in np.logspace(-12, 2.7, 37):
            ref = mp.expint(1 - a, float(t))
            got = oracle_mod.phi(a, float(t))
            worst = max(worst, float(abs(got - ref) / abs(ref)))
    assert worst < 3e-15, worst


@pytest.mark.parametrize("a", [-5.5, -3.0, -1.5, -0.5, 0.0, 0.5, 1.0, 2.5, 6.0])
def test_phi_order_recurrence(oracle_mod, a):
    # t Phi_{a+1}(t) = a Phi_a(t) + e^{-t}: integration by parts of the defining integral
    for t in [1e-3, 0.3, 0.99, 1.0, 2.0, 9.0, 40.0]:
        lhs = t * oracle_mod.phi(a + 1, t)
        rhs = a * oracle_mod.phi(a, t) + math.exp(-t)
        scale = abs(t * oracle_mod.phi(a + 1, t)) + abs(a * oracle_mod.phi(a, t)) + math.exp(-t)
        assert abs(lhs - rhs) <= 4e-15 * scale, (a, t, lhs, rhs)
