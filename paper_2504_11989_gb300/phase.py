"""Stability of fcc against bcc with two- and three-body interactions (Sec. 5).

Atoms on a Bravais lattice Lambda interact through an (n, m) Lennard-Jones potential and the
three-body Axilrod-Teller-Muto potential with coupling lambda.  With distances in units of
the equilibrium distance and energies in units of the dissociation energy, the cohesive
energy per particle of the lattice with nearest-neighbour distance R is

    E_coh(R) = n m / (2 (n - m)) (Z_{Lambda,n}(0) / (n R^n) - Z_{Lambda,m}(0) / (m R^m))
               + lambda / R^9 (zeta(3,3,3)/24 - 3 zeta(-1,5,5)/16 + 3 zeta(1,3,5)/8),

where Lambda is the lattice with unit nearest-neighbour distance, and the enthalpy per particle
at pressure p is H = E_coh + p V_Lambda R^3.  The lattice-sum work (the two Epstein zeta
values and the three three-body zeta values of each lattice) runs on the GPU through the C
ABI; what remains -- minimising H over R and locating, for each p, the coupling lambda where
the bcc enthalpy drops below the fcc one -- is a few scalar functions of R, done here on the
host in plain floating point.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# lattice matrices with unit nearest-neighbour distance, as printed in Sec. 5
UNIT_NN = ("fcc", "bcc")


@dataclass
class Coefficients:
    """Lattice sums of one lattice at unit nearest-neighbour distance."""

    name: str
    volume: float  # V_Lambda: volume per particle
    z_n: float     # Z_{Lambda,n}(0)
    z_m: float     # Z_{Lambda,m}(0)
    e_atm: float   # zeta(3,3,3)/24 - 3 zeta(-1,5,5)/16 + 3 zeta(1,3,5)/8
    n: int
    m: int


def enthalpy(c: Coefficients, lam: float, p: float, R):
    """H(R) = E_coh^(2)(R) + E_coh^(3)(R) + p V R^3 (R scalar or array)."""
    R = np.asarray(R, dtype=np.float64)
    n, m = c.n, c.m
    e2 = n * m / (2.0 * (n - m)) * (c.z_n / (n * R ** n) - c.z_m / (m * R ** m))
    return e2 + lam * c.e_atm / R ** 9 + p * c.volume * R ** 3


def enthalpy_slope(c: Coefficients, lam: float, p: float, R: float) -> float:
    """dH/dR."""
    n, m = c.n, c.m
    d2 = n * m / (2.0 * (n - m)) * (-c.z_n / R ** (n + 1) + c.z_m / R ** (m + 1))
    return d2 - 9.0 * lam * c.e_atm / R ** 10 + 3.0 * p * c.volume * R * R


def min_enthalpy(c: Coefficients, lam: float, p: float, r_lo: float = 0.6, r_hi: float = 2.0):
    """(R*, H(R*)): the minimum of H over R in [r_lo, r_hi], bracketed on a grid, then located
    as the zero of dH/dR by bisection (to the last bits of R, which the flat minimum of H
    itself would not resolve)."""
    grid = np.linspace(r_lo, r_hi, 2001)
    i = int(np.argmin(enthalpy(c, lam, p, grid)))
    a, b = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
    if enthalpy_slope(c, lam, p, a) >= 0.0 or enthalpy_slope(c, lam, p, b) <= 0.0:
        r = grid[i]  # minimum at the end of the range
        return r, float(enthalpy(c, lam, p, r))
    for _ in range(200):
        mid = 0.5 * (a + b)
        if mid <= a or mid >= b:
            break
        if enthalpy_slope(c, lam, p, mid) < 0.0:
            a = mid
        else:
            b = mid
    r = 0.5 * (a + b)
    return r, float(enthalpy(c, lam, p, r))


def enthalpy_gap(fcc: Coefficients, bcc: Coefficients, lam: float, p: float) -> float:
    """H_bcc - H_fcc at their own optimal R: > 0 where fcc is stable."""
    return min_enthalpy(bcc, lam, p)[1] - min_enthalpy(fcc, lam, p)[1]


def critical_coupling(fcc: Coefficients, bcc: Coefficients, p: float, lam_max: float = 10.0, tol: float = 1e-10):
    """The lambda in [0, lam_max] where bcc and fcc have equal enthalpy at pressure p (the
    phase boundary), by bisection on the sign of the enthalpy gap; None if fcc stays stable."""
    lo, hi = 0.0, lam_max
    g_lo, g_hi = enthalpy_gap(fcc, bcc, lo, p), enthalpy_gap(fcc, bcc, hi, p)
    if g_lo <= 0.0:
        return 0.0
    if g_hi > 0.0:
        return None
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if enthalpy_gap(fcc, bcc, mid, p) > 0.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def coefficients(ezeta, name: str, n: int, m: int, quad, stream=None) -> Coefficients:
    """The lattice sums of `name` (fcc or bcc, unit nearest-neighbour distance) through the C
    ABI: Z_n(0) and Z_m(0) by ez_epstein_zeta at y = 0 (n, m > 3, finite), the ATM energy by
    ez_atm_energy on the quadrature `quad` (an ez_quadrature)."""
    from . import workloads as W

    A = W.lattice(name, unit_density=False)
    L = ezeta.Lattice(A)
    zero = np.zeros((1, 3))
    z_n = float(ezeta.ez_epstein_zeta(L, float(n), np.zeros(3), zero, stream=stream)[0][0])
    z_m = float(ezeta.ez_epstein_zeta(L, float(m), np.zeros(3), zero, stream=stream)[0][0])
    e_atm, _ = ezeta.ez_atm_energy(L, quad, stream=stream)
    return Coefficients(name, abs(float(np.linalg.det(A))), z_n, z_m, float(e_atm), n, m)
