"""Brute-force lattice sums straight from the definitions (numpy), used only as pins.

* zeta_n_direct: Def. "Many-body zeta function" with x^(0) = x^(n) = 0, the primed sum
  dropping every summand with a vanishing distance, over A{-L..L}^d.
* atm_direct: Def. "ATM potential and cohesive energy", E = (1/6) sum' U(x, y).
* epstein_direct: Def. "Epstein zeta function" for Re nu > d, truncated at |z - x| <= R.
"""
import itertools

import numpy as np


def lattice_points(A, L):
    d = A.shape[0]
    rng = np.arange(-L, L + 1)
    m = np.array(list(itertools.product(rng, repeat=d)), dtype=np.float64)
    return m @ A.T


def epstein_direct(A, nu, x, y, R):
    d = A.shape[0]
    Ainv = np.linalg.inv(A)
    L = int(np.ceil(R * np.max(np.linalg.norm(Ainv, axis=1)))) + int(np.ceil(np.max(np.abs(Ainv @ x)))) + 1
    z = lattice_points(A, L)
    r = np.linalg.norm(z - x, axis=1)
    keep = (r > 1e-12) & (r <= R)
    z, r = z[keep], r[keep]
    ph = np.exp(-2j * np.pi * (z @ y))
    # sum smallest terms first
    order = np.argsort(-r)
    return np.sum((ph / r**nu)[order])


def zeta_n_direct(A, nus, L):
    """n in {2,3,4}: sum over x1..x_{n-1} in A{-L..L}^d of prod |x_j - x_{j-1}|^{-nu_j}."""
    pts = lattice_points(A, L)
    n = len(nus)
    if n == 2:
        r = np.linalg.norm(pts, axis=1)
        r = r[r > 1e-12]
        return float(np.sum(np.sort(r ** -(nus[0] + nus[1]))))
    total = 0.0
    r0 = np.linalg.norm(pts, axis=1)
    if n == 3:
        for i, x in enumerate(pts):
            if r0[i] < 1e-12:
                continue
            dyx = np.linalg.norm(pts - x, axis=1)
            ok = (r0 > 1e-12) & (dyx > 1e-12)
            total += r0[i] ** -nus[0] * np.sum(dyx[ok] ** -nus[1] * r0[ok] ** -nus[2])
        return total
    if n == 4:
        D = np.linalg.norm(pts[:, None, :] - pts[None, :, :], axis=2)
        with np.errstate(divide="ignore"):
            P1 = np.where(r0 > 1e-12, r0 ** -nus[0], 0.0)  # |x1|
            P4 = np.where(r0 > 1e-12, r0 ** -nus[3], 0.0)  # |x3|
            M2 = np.where(D > 1e-12, D ** -nus[1], 0.0)  # |x2 - x1|
            M3 = np.where(D > 1e-12, D ** -nus[2], 0.0)  # |x3 - x2|
        # sum_{x1,x2,x3} P1[x1] M2[x1,x2] M3[x2,x3] P4[x3]
        return float(P1 @ M2 @ M3 @ P4)
    raise ValueError(n)


def atm_direct(A, L):
    pts = lattice_points(A, L)
    r0 = np.linalg.norm(pts, axis=1)
    total = 0.0
    for i, x in enumerate(pts):
        if r0[i] < 1e-12:
            continue
        z = pts - x  # z = y - x
        rz = np.linalg.norm(z, axis=1)
        ok = (r0 > 1e-12) & (rz > 1e-12)
        y, ry, zz, rzz = pts[ok], r0[ok], z[ok], rz[ok]
        rx = r0[i]
        xy = y @ x
        yz = np.sum(y * zz, axis=1)
        zx = zz @ x
        U = (rx * ry * rzz) ** -3.0 - 3.0 * xy * yz * zx / (rx * ry * rzz) ** 5
        total += np.sum(U)
    return total / 6.0
