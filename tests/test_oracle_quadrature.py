"""Pins of the oracle's quadrature pieces: Gauss-Legendre rule (Sec. 3, tensor GL in v),
the fixed u rules, and the closed-form Hadamard integrals of Sec. 3."""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2504_11989_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 2, 3, 7, 14, 40, 100])
def test_gl_vs_numpy(oracle_mod, n):
    # numpy's leggauss weights carry ~1e-12 relative error for n ~ 40..100
    x, w = oracle_mod.gauss_legendre01(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, (xr + 1) / 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wr / 2, rtol=1e-11)


@pytest.mark.parametrize("n", [7, 40, 100])
def test_gl_vs_high_precision(oracle_mod, n):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, w = oracle_mod.gauss_legendre01(n)

    def legendre(z):
        p0, p1 = mp.mpf(1), z
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * z * p1 - (k - 1) * p0) / k
        return p1, p0

    for i in range(n):
        z = mp.mpf(1 - 2 * x[i])
        for _ in range(8):
            pn, pm = legendre(z)
            z -= pn / (n * (z * pn - pm) / (z * z - 1))
        pn, pm = legendre(z)
        dp = n * (z * pn - pm) / (z * z - 1)
        assert abs(x[i] - float((1 - z) / 2)) <= 2.3e-16  # one ulp
        assert w[i] == pytest.approx(float(1 / ((1 - z * z) * dp * dp)), rel=3e-14)


@pytest.mark.parametrize("n", [64, 512, 4096])
def test_gl_exact_on_polynomials(oracle_mod, n):
    x, w = oracle_mod.gauss_legendre01(n)
    for k in [0, 1, 5, 17, 2 * n - 1]:
        # int_0^1 x^k dx = 1/(k+1)
        assert float(np.sum(w * x**k)) == pytest.approx(1.0 / (k + 1), rel=1e-13)
    assert np.all(np.diff(x) > 0)


def test_u_rules_cover_interval(oracle_mod):
    p1 = W.nbody_problem("Z", 4.0, 3, W.Quad(n_u=33, n_v=1, u_rule=1))
    u, w = oracle_mod.u_rule(p1)
    assert u.size == 33 and np.sum(w) == pytest.approx(0.5, rel=1e-15)
    assert np.all((u > 0) & (u < 0.5))
    p2 = W.atm_problem("Z", W.Quad(n_u=9, n_v=1, u_rule=2, eps=1e-2))
    u, w = oracle_mod.u_rule(p2)
    assert u.size == 6 * 9  # panels [.01,.02] .. [.32,.5]
    assert np.sum(w) == pytest.approx(0.5 - 1e-2, rel=1e-15)
    assert np.all((u > 1e-2) & (u < 0.5))
    # graded panels integrate u^{-1/2} log u accurately (singularity outside)
    ref = integrate.quad(lambda t: t**-0.5 * math.log(t), 1e-2, 0.5, epsrel=1e-14)[0]
    assert float(np.sum(w * u**-0.5 * np.log(u))) == pytest.approx(ref, rel=1e-12)


PRINTED = {
    # closed forms printed in Sec. 3 for m = 0..3 (L = log(pi eps^2 w^2))
    0: lambda mu, e, L: e**mu / mu,
    1: lambda mu, e, L: -e**mu * (2 - mu * L) / mu**2,
    2: lambda mu, e, L: e**mu * (8 - mu * L * (4 - mu * L)) / mu**3,
    3: lambda mu, e, L: -e**mu * (48 - mu * L * (24 - mu * L * (6 - mu * L))) / mu**4,
}


@pytest.mark.parametrize("m", [0, 1, 2, 3])
@pytest.mark.parametrize("mu", [-3.0, -1.0, 0.5, 1.0, 3.0, 7.0])
def test_hadamard_vs_printed_closed_forms(oracle_mod, m, mu):
    eps, w2 = 1e-2, 1.7
    L = math.log(math.pi * eps * eps * w2)
    assert oracle_mod.hadamard(mu, m, eps, w2) == pytest.approx(PRINTED[m](mu, eps, L), rel=1e-13)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mu", [1.0, 2.5, 5.0])
def test_hadamard_vs_numerical_integral(oracle_mod, m, mu):
    eps, w2 = 0.05, 0.8
    f = lambda u: u ** (mu - 1) * math.log(math.pi * u * u * w2) ** m
    ref = integrate.quad(f, 0.0, eps, epsabs=0, epsrel=1e-13, limit=500)[0]
    assert oracle_mod.hadamard(mu, m, eps, w2) == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("m", [0, 1, 2])
def test_hadamard_finite_part_for_negative_mu(oracle_mod, m):
    # finite part for mu < 0: int_delta^eps u^{mu-1} L^m du minus its divergent
    # part as delta -> 0, which is exactly -I_m evaluated at the lower limit delta
    mu, eps, w2, delta = -1.0, 0.1, 1.3, 1e-3
    f = lambda u: u ** (mu - 1) * math.log(math.pi * u * u * w2) ** m
    num = integrate.quad(f, delta, eps, epsabs=0, epsrel=1e-13, limit=500)[0]
    at_delta = oracle_mod.hadamard(mu, m, delta, w2)
    assert oracle_mod.hadamard(mu, m, eps, w2) == pytest.approx(num + at_delta, rel=1e-10)


def test_gl_endpoint_nodes_relative_accuracy(oracle_mod):
    # nodes next to the endpoints of a 4096-point rule (the config-1 u rule) must be
    # accurate relative to their own size, not just to 1e-16 absolute
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    n = 4096
    x, w = oracle_mod.gauss_legendre01(n)

    def legendre(z):
        p0, p1 = mp.mpf(1), z
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * z * p1 - (k - 1) * p0) / k
        return p1, p0

    for i in (0, 1, 5, n - 2, n - 1):
        z = 1 - 2 * mp.mpf(x[i])
        for _ in range(4):
            pn, pm = legendre(z)
            z -= pn / (n * (z * pn - pm) / (z * z - 1))
        pn, pm = legendre(z)
        dp = n * (z * pn - pm) / (z * z - 1)
        assert x[i] == pytest.approx(float((1 - z) / 2), rel=4e-15)
        assert w[i] == pytest.approx(float(1 / ((1 - z * z) * dp * dp)), rel=8e-15)
