"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds no arithmetic of the method: only lattice matrices (as printed
in the paper), unit-density rescaling of those matrices, quadrature-size presets
and seeded random draws (lattice constants, request mixes, Poisson arrivals).

Lattice matrices (columns are the basis vectors, Lambda = A Z^d):
  * Z, square, simple cubic: identity.
  * hexagonal A_hex: Sec. 4.1 ("Error scaling with numerical discretization
    parameters"), the matrix [[1, 1/2], [0, sqrt(3)/2]].
  * A_kappa (condition number kappa): Eq. (A_kappa), Sec. 4.1.
  * fcc / bcc: Sec. 4.1 and again Sec. 5 (unit nearest-neighbour distance).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20261203


def _a_kappa(kappa: float) -> np.ndarray:
    return np.array([[1.0, (kappa - 1.0 / kappa) / 2.0], [0.0, (kappa + 1.0 / kappa) / 2.0]])


_S2 = math.sqrt(2.0)
_S3 = math.sqrt(3.0)

PRESETS = {
    "Z": np.array([[1.0]]),
    "square": np.eye(2),
    "hexagonal": np.array([[1.0, 0.5], [0.0, _S3 / 2.0]]),
    "sc": np.eye(3),
    "fcc": np.array([[1.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 1.0]]) / _S2,
    "bcc": np.array([[1.0, 1.0, 0.0], [_S2, 0.0, _S2], [0.0, _S2, _S2]]) / _S3,
}



def _from_gram(G) -> np.ndarray:
    """A basis with Gram matrix G (A^T A = G): the transposed Cholesky factor."""
    return np.linalg.cholesky(np.asarray(G, dtype=np.float64)).T


def _cartan(n: int, edges) -> np.ndarray:
    """Cartan matrix of a simply laced Dynkin diagram: 2 on the diagonal, -1 per edge."""
    G = 2.0 * np.eye(n)
    for i, j in edges:
        G[i, j] = G[j, i] = -1.0
    return G


# higher dimensions (the Epstein zeta function alone): cubic lattices, the root lattices D4
# (densest packing in four dimensions), D5 and E6, given by the Gram matrices of their
# simple roots
PRESETS.update({
    "Z4": np.eye(4),
    "D4": _from_gram(_cartan(4, [(0, 1), (1, 2), (1, 3)])),
    "Z5": np.eye(5),
    "D5": _from_gram(_cartan(5, [(0, 1), (1, 2), (2, 3), (2, 4)])),
    "Z6": np.eye(6),
    "E6": _from_gram(_cartan(6, [(0, 2), (2, 3), (3, 4), (4, 5), (1, 3)])),
})

DIM_OF = {"Z": 1, "square": 2, "hexagonal": 2, "sc": 3, "fcc": 3, "bcc": 3, "Z4": 4, "D4": 4, "Z5": 5, "D5": 5,
          "Z6": 6, "E6": 6}
LATTICES_BY_DIM = {1: ["Z"], 2: ["square", "hexagonal"], 3: ["sc", "fcc", "bcc"], 4: ["Z4", "D4"], 5: ["Z5", "D5"],
                   6: ["Z6", "E6"]}


def lattice(name: str, unit_density: bool = True, scale: float = 1.0) -> np.ndarray:
    """Row-major d x d matrix A (A[i, j] = component i of basis vector j).

    unit_density rescales A so that |det A| = 1; scale multiplies afterwards
    (the lattice constant of the served stability scan).
    """
    if name.startswith("kappa="):
        a = _a_kappa(float(name.split("=", 1)[1]))
    else:
        a = PRESETS[name].copy()
    if unit_density:
        d = a.shape[0]
        a = a / abs(np.linalg.det(a)) ** (1.0 / d)
    return np.ascontiguousarray(a * scale, dtype=np.float64)


@dataclass
class Quad:
    """Quadrature/truncation parameters of one lattice sum (mirrors ez_quadrature).

    u_rule: 1 = one Gauss-Legendre rule with n_u nodes on [0, 1/2];
            2 = eps-split: analytic near part on [0, eps] plus graded panels
                [eps, 2 eps], [2 eps, 4 eps], ... , [., 1/2] with n_u nodes each.
    """

    n_u: int
    n_v: int
    u_rule: int = 1
    eps: float = 1e-2
    ell: int = 4
    lam: float = 1.0
    r_real: float = 6.0
    r_recip: float = 6.0


@dataclass
class Problem:
    name: str
    A: np.ndarray
    nu: list  # distinct exponents
    expo: list  # per product: exponent count per distinct nu
    quad: Quad
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return self.A.shape[0]


ATM_NU = [-1.0, 1.0, 3.0, 5.0]
# products (3,3,3), (-1,5,5), (1,3,5) over the distinct list ATM_NU
ATM_EXPO = [[0, 0, 3, 0], [1, 0, 0, 2], [0, 1, 1, 1]]


def nbody_problem(lat: str, nu: float, n: int, quad: Quad, scale: float = 1.0) -> Problem:
    return Problem(f"{lat}:nu={nu}:n={n}", lattice(lat, scale=scale), [float(nu)], [[n]], quad)


def atm_problem(lat: str, quad: Quad, scale: float = 1.0) -> Problem:
    return Problem(f"{lat}:ATM", lattice(lat, scale=scale), list(ATM_NU), [list(r) for r in ATM_EXPO], quad)


def config1(n_u: int = 4096) -> Quad:
    """d=1, Lambda=Z, nu=(4,4,4): 4096 GL nodes on [0,1/2], 8 shells each side."""
    return Quad(n_u=n_u, n_v=1, u_rule=1, lam=1.0, r_real=8.0, r_recip=8.0)


def config2(n: int = 256) -> Quad:
    """d=2, tensor grid n x n mapped to 4 Duffy sectors x (n/2) u-nodes x (n/2) v-nodes."""
    return Quad(n_u=n // 2, n_v=n // 2, u_rule=1, lam=1.0, r_real=6.0, r_recip=6.0)


def config3(n_v: int = 64, n_u_panel: int = 8) -> Quad:
    """d=3 ATM: eps-split with 6 graded panels; n_v GL nodes per v axis."""
    return Quad(n_u=n_u_panel, n_v=n_v, u_rule=2, eps=1e-2, ell=4, lam=1.0, r_real=4.5, r_recip=4.5)


def config4(n_v: int = 48, n_u: int = 32) -> Quad:
    """d=3 fcc, nu=6 chain sums: 12 sectors x n_u x n_v^2 nodes."""
    return Quad(n_u=n_u, n_v=n_v, u_rule=1, lam=1.0, r_real=4.5, r_recip=4.5)


def explicit_splitting(prob: Problem, shells: float = 6.0) -> Problem:
    """Copy of `prob` whose automatic splitting parameter and cutoffs (lam = 0, r = 0)
    are replaced by explicit ones: lam = V^{1/d}, r_real = shells lam, r_recip = shells / lam.
    The lattice sum does not depend on lam; the oracle needs explicit values."""
    q = prob.quad
    if q.lam > 0.0 and q.r_real > 0.0 and q.r_recip > 0.0:
        return prob
    lam = q.lam if q.lam > 0.0 else abs(float(np.linalg.det(prob.A))) ** (1.0 / prob.d)
    q2 = Quad(q.n_u, q.n_v, q.u_rule, q.eps, q.ell, lam, shells * lam, shells / lam)
    return Problem(prob.name, prob.A, prob.nu, prob.expo, q2, dict(prob.meta))


def lattice_constants(count: int, seed: int, lo: float = 0.9, hi: float = 1.3) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=count)


@dataclass
class Request:
    rid: int
    arrival_s: float
    d: int
    lattice: str
    scale: float
    kind: str  # "nbody" or "atm"
    nu: float
    n: int
    res: int  # BZ resolution per axis


def serving_mix(count: int, seed: int, rate_per_s: float) -> list:
    """Stability-scan request stream: Poisson arrivals, random d, lattice, constant,
    exponent (or the ATM form), n and BZ resolution per axis (d=3 capped at 128)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    out = []
    for i in range(count):
        d = int(rng.integers(1, 4))
        lat = LATTICES_BY_DIM[d][int(rng.integers(0, len(LATTICES_BY_DIM[d])))]
        scale = float(rng.uniform(0.9, 1.3))
        pick = int(rng.integers(0, 5))
        kind = "atm" if pick == 4 else "nbody"
        nu = [4.0, 6.0, 9.0, 12.0][pick] if pick < 4 else 0.0
        n = 3 if kind == "atm" else int(rng.integers(2, 4))
        resopts = [64, 96, 128, 192, 256]
        res = resopts[int(rng.integers(0, 5))]
        if d == 3:
            res = min(res, 128)
        out.append(Request(i, float(t[i]), d, lat, scale, kind, nu, n, res))
    return out


def serve_quad(d: int, res: int, singular: bool, lam: float = 0.0) -> Quad:
    """Quadrature of a served request at BZ resolution `res` per axis: n_v = res/2 per v
    axis; n_u from the node budget res^d / (sectors n_v^{d-1}) (d = 1: res nodes on [0,1/2]);
    the eps-split rule spreads n_u over its six graded panels.  Cutoffs from the default
    tolerance (lam = 0: lam = V^{1/d})."""
    n_v = max(2, res // 2)
    if d == 1:
        n_u = res
    elif d == 2:
        n_u = res // 2
    else:
        n_u = -(-res ** 3 // (12 * n_v * n_v))
    if singular:
        return Quad(n_u=max(4, -(-n_u // 6)), n_v=n_v, u_rule=2, lam=lam, r_real=0.0, r_recip=0.0)
    return Quad(n_u=n_u, n_v=n_v, u_rule=1, lam=lam, r_real=0.0, r_recip=0.0)


def request_problem(r: "Request") -> Problem:
    """The lattice sum of one served request."""
    A = lattice(r.lattice, scale=r.scale)
    if r.kind == "atm":
        singular = True
        nu, expo = list(ATM_NU), [list(x) for x in ATM_EXPO]
    else:
        nu, expo = [float(r.nu)], [[r.n]]
        dn = int(r.nu) - r.d
        singular = dn < 0 or dn % 2 == 0
    return Problem(f"req{r.rid}", A, nu, expo, serve_quad(r.d, r.res, singular), {"request": r})
