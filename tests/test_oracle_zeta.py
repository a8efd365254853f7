"""Pins of the oracle's Epstein zeta function Z_{Lambda,nu}(x, y) (Def. "Epstein zeta
function", incomplete-gamma splitting) and of its singular split (Sec. 3).

Independent references: Bernoulli-polynomial Fourier series (d=1, even nu), the
log and negative-exponent continuations on Z, Riemann/Hurwitz zeta, 4 zeta(s) beta(s)
for the square lattice, a theta-function integral for Z^3, brute-force sums for
large nu at arbitrary (x, y), invariance under the splitting parameter and the
lattice basis, quasi-periodicity, and the 1-D Taylor expansion of Sec. 4.3 read as
Z_{Z,nu}(k) = s_hat_nu(k) + sum_n (-1)^n (2 pi k)^{2n}/(2n)! * 2 zeta(nu - 2n).
"""
import math

import numpy as np
import pytest
from scipy import special

from paper_2504_11989_gb300 import workloads as W
from tests import brute

Z1 = np.array([[1.0]])


BERNOULLI = {  # textbook Bernoulli polynomials
    2: lambda x: x * x - x + 1.0 / 6.0,
    4: lambda x: x**4 - 2 * x**3 + x * x - 1.0 / 30.0,
    6: lambda x: x**6 - 3 * x**5 + 2.5 * x**4 - 0.5 * x * x + 1.0 / 42.0,
}


def bernoulli_poly(n, x):
    return BERNOULLI[n](x)


@pytest.mark.parametrize("s", [1, 2, 3])
@pytest.mark.parametrize("lam", [0.7, 1.0, 1.4])
def test_z_bernoulli_even_nu(oracle_mod, s, lam):
    # Z_{Z,2s}(k) = 2 sum_n cos(2 pi n k)/n^{2s} = (-1)^{s+1} (2 pi)^{2s} B_{2s}(k) / (2s)!
    for k in [0.0, 0.05, 0.2, 0.37, 0.5, 0.81]:
        ref = (-1) ** (s + 1) * (2 * math.pi) ** (2 * s) * bernoulli_poly(2 * s, k) / math.factorial(2 * s)
        z = oracle_mod.epstein_zeta(Z1, 2 * s, [0], [k], lam, 9, 9)
        assert z.real == pytest.approx(ref, rel=5e-14, abs=2e-14)
        assert abs(z.imag) < 1e-15


def test_z_log_and_negative_continuations(oracle_mod):
    for k in [0.03, 0.17, 0.3, 0.5]:
        s2 = math.sin(math.pi * k) ** 2
        assert oracle_mod.epstein_zeta(Z1, 1.0, [0], [k], 1.0, 9, 9).real == pytest.approx(-math.log(4 * s2), rel=1e-14, abs=1e-15)
        assert oracle_mod.epstein_zeta(Z1, -1.0, [0], [k], 1.0, 9, 9).real == pytest.approx(-1 / (2 * s2), rel=1e-14)


@pytest.mark.parametrize("nu", [2.0, 3.0, 4.0, 5.0, 9.0])
def test_z_at_zero_is_2zeta(oracle_mod, nu):
    assert oracle_mod.epstein_zeta(Z1, nu, [0], [0], 1.0, 9, 9).real == pytest.approx(2 * special.zeta(nu), rel=2e-15)


@pytest.mark.parametrize("x", [0.1, 0.3, 0.77])
def test_z_hurwitz(oracle_mod, x):
    for nu in [2.0, 3.0, 6.0]:
        ref = special.zeta(nu, x) + special.zeta(nu, 1 - x)
        assert oracle_mod.epstein_zeta(Z1, nu, [x], [0], 1.0, 9, 9).real == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("nu", [3.0, 5.0, 6.0, 9.0])
def test_square_lattice_zeta_beta(oracle_mod, nu):
    s = nu / 2
    beta = 4 ** -s * (special.zeta(s, 0.25) - special.zeta(s, 0.75))
    ref = 4 * special.zeta(s) * beta
    assert oracle_mod.epstein_zeta(np.eye(2), nu, [0, 0], [0, 0], 1.0, 7, 7).real == pytest.approx(ref, rel=1e-14)


def test_simple_cubic_theta_integral(oracle_mod):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 25
    nu = 6
    # theta_3(e^{-pi t}) = t^{-1/2} theta_3(e^{-pi/t}) (Jacobi) keeps the nome small for t < 1
    def th3(t):
        if t < 1:
            return mp.jtheta(3, 0, mp.exp(-mp.pi / t)) / mp.sqrt(t)
        return mp.jtheta(3, 0, mp.exp(-mp.pi * t))

    f = lambda t: t ** (nu / 2 - 1) * (th3(t) ** 3 - 1)
    ref = float(mp.pi ** (nu / 2) / mp.gamma(nu / 2) * mp.quad(f, [0, 1, mp.inf]))
    assert oracle_mod.epstein_zeta(np.eye(3), nu, [0] * 3, [0] * 3, 1.0, 5, 5).real == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("lat", ["hexagonal", "fcc", "kappa=2"])
def test_general_xy_vs_brute_force(oracle_mod, lat):
    rng = np.random.default_rng(7)
    A = W.lattice(lat)
    d = A.shape[0]
    nu = 14.0 if d == 3 else 16.0
    for _ in range(3):
        x = A @ rng.uniform(-0.5, 0.5, d)
        y = np.linalg.inv(A).T @ rng.uniform(-0.5, 0.5, d)
        ref = brute.epstein_direct(A, nu, x, y, 12.0)
        got = oracle_mod.epstein_zeta(A, nu, x, y, 1.0, 8, 8)
        assert abs(got - ref) <= 1e-13 * abs(ref)


@pytest.mark.parametrize("lat,nu", [("square", -1.0), ("hexagonal", 3.0), ("fcc", 1.0), ("bcc", 5.0), ("fcc", 6.0)])
def test_lambda_invariance(oracle_mod, lat, nu):
    A = W.lattice(lat)
    d = A.shape[0]
    rng = np.random.default_rng(3)
    for _ in range(3):
        k = np.linalg.inv(A).T @ rng.uniform(-0.5, 0.5, d)
        x = A @ rng.uniform(-0.5, 0.5, d)
        vals = [oracle_mod.epstein_zeta(A, nu, x, k, lam, 9.0, 9.0) for lam in (0.8, 1.0, 1.25)]
        for v in vals[1:]:
            assert abs(v - vals[0]) <= 1e-13 * max(1.0, abs(vals[0]))


def test_quasi_periodicity_and_basis_invariance(oracle_mod):
    A = W.lattice("hexagonal")
    x, y = np.array([0.21, 0.11]), np.array([0.13, -0.31])
    z0 = A @ np.array([1, -2])
    g0 = np.linalg.inv(A).T @ np.array([2, 1])
    base = oracle_mod.epstein_zeta(A, 5.0, x, y, 1.0, 8, 8)
    assert oracle_mod.epstein_zeta(A, 5.0, x + z0, y, 1.0, 8, 8) == pytest.approx(base * np.exp(-2j * np.pi * (y @ z0)), rel=1e-13)
    assert oracle_mod.epstein_zeta(A, 5.0, x, y + g0, 1.0, 8, 8) == pytest.approx(base, rel=1e-13)
    U = np.array([[1, 1], [0, 1]])  # unimodular change of basis
    c, s = math.cos(0.3), math.sin(0.3)
    Q = np.array([[c, -s], [s, c]])
    A2 = Q @ A @ U
    assert oracle_mod.epstein_zeta(A2, 5.0, Q @ x, Q @ y, 1.0, 8, 8) == pytest.approx(base, rel=1e-13)


@pytest.mark.parametrize("nu", [4.0, 6.0, -1.0, 2.0, -3.0])
def test_d1_taylor_coefficients_of_zreg(oracle_mod, nu):
    """Sec. 4.3, 1-D expansion (read as (-1)^n (2 pi k)^{2n}/(2n)! * Z_{nu-2n}(0), Z_{Z,s}(0) = 2 zeta(s))."""
    mp = pytest.importorskip("mpmath")
    prob = W.Problem("z", Z1, [nu], [[1]], W.Quad(n_u=4, n_v=1, ell=6, lam=1.0, r_real=9, r_recip=9))
    C = oracle_mod.reg_taylor(prob, 0, [1.0])
    for n in range(7):
        ref = (-1) ** n * (2 * math.pi) ** (2 * n) / math.factorial(2 * n) * 2 * float(mp.zeta(nu - 2 * n))
        scale = max(1.0, (2 * math.pi) ** (2 * n) / math.factorial(2 * n))  # cancellation grows like this
        assert C[n] == pytest.approx(ref, rel=1e-12, abs=1e-13 * scale * abs(C[0]))


@pytest.mark.parametrize("lat,nu", [("square", 3.0), ("hexagonal", -1.0), ("fcc", 5.0), ("bcc", 1.0), ("sc", 3.0)])
def test_zreg_direct_vs_taylor(oracle_mod, lat, nu):
    # Z^reg computed as Z - s_hat/V (Crandall + Sec. 3 singularity) agrees with its own
    # Taylor polynomial built term by term (different code path) at |k| ~ 0.02
    A = W.lattice(lat)
    d = A.shape[0]
    prob = W.Problem("z", A, [nu], [[1]], W.Quad(n_u=4, n_v=4, ell=6, lam=1.0, r_real=8, r_recip=8))
    rng = np.random.default_rng(11)
    for _ in range(3):
        w = rng.normal(size=d)
        w /= np.linalg.norm(w)
        C = oracle_mod.reg_taylor(prob, 0, w)
        for u in [0.005, 0.02, 0.06]:
            direct = oracle_mod.epstein_zeta_reg(A, nu, u * w, 1.0, 8, 8)
            series = sum(C[k] * u ** (2 * k) for k in range(len(C)))
            # Z - s_hat/V cancels the singular term: allow rounding at its size
            sing = abs(oracle_mod.s_hat(d, nu, u * w)) / abs(np.linalg.det(A))
            assert direct == pytest.approx(series, rel=1e-12, abs=1e-12 + 1e-14 * sing)


# ----------------------------------------------------------------- real (non-integer) exponents
@pytest.mark.parametrize("nu", [1.5, 2.3, 3.7, 4.25, 7.9])
def test_real_nu_d1_closed_forms(oracle_mod, nu):
    # Z(0) = 2 zeta(nu); Z(x, 0) = zeta(nu, x) + zeta(nu, 1 - x) (Hurwitz); and at y != 0 the
    # periodic zeta function 2 Re Li_nu(e^{2 pi i y}) (mpmath, 30 digits)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    assert oracle_mod.epstein_zeta(Z1, nu, [0], [0], 1.0, 9, 9).real == pytest.approx(2 * special.zeta(nu), rel=3e-15)
    for x in (0.15, 0.6):
        ref = special.zeta(nu, x) + special.zeta(nu, 1 - x)
        assert oracle_mod.epstein_zeta(Z1, nu, [x], [0], 1.0, 9, 9).real == pytest.approx(ref, rel=2e-14)
    for y in (0.07, 0.31, 0.5):
        ref = float(2 * mp.re(mp.polylog(nu, mp.exp(2j * mp.pi * y))))
        z = oracle_mod.epstein_zeta(Z1, nu, [0], [y], 1.2, 9, 9)
        assert z.real == pytest.approx(ref, rel=1e-13, abs=1e-14), (nu, y)


@pytest.mark.parametrize("lat,nu", [("hexagonal", 3.4), ("fcc", 5.5), ("square", -0.6)])
def test_real_nu_lambda_invariance(oracle_mod, lat, nu):
    A = W.lattice(lat)
    d = A.shape[0]
    y = np.linalg.inv(A).T @ (np.arange(1, d + 1) * 0.137)
    za = oracle_mod.epstein_zeta(A, nu, np.zeros(d), y, 0.8, 9 * 0.8, 9 / 0.8)
    zb = oracle_mod.epstein_zeta(A, nu, np.zeros(d), y, 1.3, 9 * 1.3, 9 / 1.3)
    assert abs(za - zb) <= 2e-14 * max(1.0, abs(za))


def test_real_nu_lattice_sums(oracle_mod):
    # Cor. one/two-body: zeta^(2)(nu1, nu2) = Z_{nu1+nu2}(0) and zeta^(1) = 0 for real exponents
    # (the u integral takes the eps-split, nu - d not an odd integer); three-body against the
    # direct sum at large exponents (d = 1)
    for lat, nus in (("square", (2.7, 3.6)), ("Z", (1.8, 2.45))):
        A = W.lattice(lat)
        d = A.shape[0]
        q = W.Quad(n_u=16, n_v=16 if d == 2 else 1, u_rule=2, lam=1.0, r_real=7.0, r_recip=7.0)
        two = oracle_mod.nbody(W.Problem("z", A, list(nus), [[1, 1]], q), threads=8)[0]
        ref = oracle_mod.epstein_zeta(A, sum(nus), np.zeros(d), np.zeros(d), 1.0, 9, 9).real
        assert two == pytest.approx(ref, rel=1e-13)
        one = oracle_mod.nbody(W.Problem("z", A, [nus[0]], [[1]], q), threads=8)[0]
        assert abs(one) < 1e-13
    nus = (6.3, 7.1, 8.6)
    prob = W.Problem("z", Z1, list(nus), [[1, 1, 1]], W.Quad(n_u=8, n_v=1, u_rule=2, lam=1.0, r_real=9, r_recip=9))
    assert oracle_mod.nbody(prob)[0] == pytest.approx(brute.zeta_n_direct(Z1, nus, 600), rel=2e-14)


# ----------------------------------------------------------------- dimensions d = 4, 5, 6
@pytest.mark.parametrize("s", [2.5, 3.0, 4.5])
def test_nd_z4_jacobi_four_squares(oracle_mod, s):
    # sum' |m|^{-2s} over Z^4 = sum_n r_4(n) n^{-s} = 8 (1 - 4^{1-s}) zeta(s) zeta(s-1) (Jacobi)
    ref = 8 * (1 - 4 ** (1 - s)) * special.zeta(s) * special.zeta(s - 1)
    z = oracle_mod.epstein_zeta_nd(np.eye(4), 2 * s, np.zeros(4), np.zeros(4), 1.0, 7.0, 7.0)
    assert z.real == pytest.approx(ref, rel=1e-14) and abs(z.imag) < 1e-14


@pytest.mark.parametrize("d,nu", [(5, 8.0), (6, 9.0), (4, 7.3)])
def test_nd_zd_theta_integral(oracle_mod, d, nu):
    # Z_{Z^d,nu}(0) = pi^{nu/2} / Gamma(nu/2) int_0^inf t^{nu/2-1} (theta_3(e^{-pi t})^d - 1) dt
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 25
    def th(t):  # theta_3(e^{-pi t}), by the Jacobi transformation t^{-1/2} theta_3(e^{-pi/t}) for t < 1
        return mp.jtheta(3, 0, mp.exp(-mp.pi * t)) if t >= 1 else mp.jtheta(3, 0, mp.exp(-mp.pi / t)) / mp.sqrt(t)

    f = lambda t: t ** (nu / 2 - 1) * (th(t) ** d - 1)
    ref = float(mp.pi ** (nu / 2) / mp.gamma(nu / 2) * mp.quad(f, [0, 1, mp.inf]))
    z = oracle_mod.epstein_zeta_nd(np.eye(d), nu, np.zeros(d), np.zeros(d), 1.0, 7.0, 7.0)
    assert z.real == pytest.approx(ref, rel=1e-13)


D4_SKEW = np.array([[1.0, 0.2, 0.0, -0.1], [0.0, 1.1, 0.3, 0.0], [0.1, 0.0, 0.9, 0.2], [0.0, -0.2, 0.1, 1.05]])


@pytest.mark.parametrize("nu", [3.0, 6.5, -1.5])
def test_nd_lambda_invariance(oracle_mod, nu):
    d = 4
    x = D4_SKEW @ np.array([0.13, -0.27, 0.4, 0.05])
    y = np.linalg.inv(D4_SKEW).T @ np.array([0.21, -0.33, 0.12, 0.44])
    za = oracle_mod.epstein_zeta_nd(D4_SKEW, nu, x, y, 0.85, 7 * 0.85, 7 / 0.85)
    zb = oracle_mod.epstein_zeta_nd(D4_SKEW, nu, x, y, 1.25, 7 * 1.25, 7 / 1.25)
    assert abs(za - zb) <= 3e-14 * max(1.0, abs(za))


def test_nd_brute_force_and_lower_dimensions(oracle_mod):
    # large nu: the defining sum sum_z e^{-2 pi i y.z} |z - x|^{-nu} directly (d = 4)
    nu, d, L = 18.0, 4, 5
    x = D4_SKEW @ np.array([0.3, 0.1, -0.2, 0.15])
    y = np.array([0.1, 0.25, -0.3, 0.05])
    g = np.array(np.meshgrid(*[np.arange(-L, L + 1)] * d, indexing="ij")).reshape(d, -1).T
    z = g @ D4_SKEW.T
    r = np.linalg.norm(z - x, axis=1)
    ref = np.sum(np.exp(-2j * np.pi * (z @ y)) * r ** -nu)
    got = oracle_mod.epstein_zeta_nd(D4_SKEW, nu, x, y, 1.0, 7.0, 7.0)
    assert abs(got - ref) <= 1e-13 * abs(ref)
    # d <= 3: the same values as the three-dimensional oracle
    for lat in ("Z", "hexagonal", "fcc"):
        A = W.lattice(lat)
        dd = A.shape[0]
        xv, yv = A @ (0.2 * np.ones(dd)), 0.17 * np.ones(dd)
        assert oracle_mod.epstein_zeta_nd(A, 3.7, xv, yv, 1.0, 8, 8) == pytest.approx(
            oracle_mod.epstein_zeta(A, 3.7, xv, yv, 1.0, 8, 8), rel=1e-15, abs=1e-15)
