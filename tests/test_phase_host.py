"""Host logic of the fcc/bcc stability scan (Sec. 5): enthalpy minimisation over the
nearest-neighbour distance and the critical ATM coupling, pinned by closed forms on
synthetic coefficients and, at zero three-body coupling, by the classical result that the
Lennard-Jones fcc lattice is more stable than bcc (lattice sums from the oracle)."""
import math

import numpy as np
import pytest

from paper_2504_11989_gb300 import phase as P
from paper_2504_11989_gb300 import workloads as W


def _synthetic(name, z_n, z_m, e_atm, volume, n=12, m=6):
    return P.Coefficients(name, volume, z_n, z_m, e_atm, n, m)


@pytest.mark.parametrize("n,m", [(12, 6), (8, 4)])
def test_pure_lennard_jones_minimum(n, m):
    # lambda = p = 0: dE/dR = 0 at R*^(n-m) = z_n / z_m, and E(R*) = -(z_m^n / z_n^m)^(1/(n-m)) / 2
    c = _synthetic("x", 12.5, 14.0, 3.0, 0.7, n, m)
    r, h = P.min_enthalpy(c, 0.0, 0.0)
    r_exact = (c.z_n / c.z_m) ** (1.0 / (n - m))
    assert r == pytest.approx(r_exact, rel=1e-9)
    assert h == pytest.approx(-0.5 * (c.z_m ** n / c.z_n ** m) ** (1.0 / (n - m)), rel=1e-12)


def test_minimum_is_stationary_with_pressure_and_three_body():
    c = _synthetic("x", 12.1, 14.4, 19.0, 0.707)
    for lam, p in ((0.3, 0.0), (0.8, 2.0), (2.0, 5.0)):
        r, h = P.min_enthalpy(c, lam, p)
        e = 1e-5
        d = (P.enthalpy(c, lam, p, r + e) - P.enthalpy(c, lam, p, r - e)) / (2 * e)
        assert abs(P.enthalpy_slope(c, lam, p, r)) < 1e-12, (lam, p, d)
        assert abs(d) < 1e-6, (lam, p, d)
        assert all(P.enthalpy(c, lam, p, r * f) > h for f in (0.98, 1.02))


def test_critical_coupling_brackets_the_crossing():
    # bcc: higher two-body energy but lower three-body energy than fcc, so a crossing exists
    f = _synthetic("fcc", 12.13, 14.45, 19.2, 0.7071)
    b = _synthetic("bcc", 9.11, 12.25, 14.8, 0.7698)
    lam_c = P.critical_coupling(f, b, 1.0)
    assert lam_c is not None and 0.0 < lam_c < 10.0
    assert P.enthalpy_gap(f, b, lam_c - 1e-6, 1.0) > 0.0 > P.enthalpy_gap(f, b, lam_c + 1e-6, 1.0)
    # without a crossing in range
    assert P.critical_coupling(f, _synthetic("b", 9.11, 12.25, 30.0, 0.7698), 1.0) is None


@pytest.mark.parametrize("n,m", [(12, 6), (8, 4)])
def test_fcc_is_stable_without_three_body_forces(oracle_mod, n, m):
    # Sec. 5: for vanishing lambda the fcc phase is always favourable (classical Lennard-Jones
    # result); Z_{Lambda,n}(0) from the oracle for the unit-nearest-neighbour lattices
    coef = {}
    for name in P.UNIT_NN:
        A = W.lattice(name, unit_density=False)
        lam = abs(np.linalg.det(A)) ** (1.0 / 3.0)
        z = {nu: oracle_mod.epstein_zeta(A, float(nu), np.zeros(3), np.zeros(3), lam, 8 * lam, 8 / lam).real
             for nu in (n, m)}
        coef[name] = P.Coefficients(name, abs(np.linalg.det(A)), z[n], z[m], 0.0, n, m)
    # every lattice vector of A_fcc / A_bcc has length >= 1, twelve (fcc) and eight (bcc) equal 1
    for name, count in (("fcc", 12), ("bcc", 8)):
        A = W.lattice(name, unit_density=False)
        r = sorted(np.linalg.norm(A @ np.array(v)) for v in np.ndindex(5, 5, 5) if any(v))
        pts = [np.linalg.norm(A @ (np.array(v) - 2)) for v in np.ndindex(5, 5, 5) if any(np.array(v) - 2)]
        assert min(pts) == pytest.approx(1.0, rel=1e-14)
        assert sum(1 for x in pts if abs(x - 1.0) < 1e-12) == count
    for p in (0.0, 1.0, 5.0):
        assert P.enthalpy_gap(coef["fcc"], coef["bcc"], 0.0, p) > 0.0
