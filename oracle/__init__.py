"""Plain FP64 CPU oracle for the Epstein zeta method (Buchheit & Busse).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2504_11989_gb300``) never imports it, and
the two share no code: the C sources here are compiled into their own library
(``oracle/_build/libezoracle.so``) by :func:`build`.

What each function follows in the paper is stated in ``ezoracle.c``; the
recombination of the ATM energy follows the Proposition of Sec. 2
(E = zeta(3,3,3)/24 - 3 zeta(-1,5,5)/16 + 3 zeta(1,3,5)/8).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library special functions, brute-force lattice sums
and values printed in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libezoracle.so")
_SRC = os.path.join(_HERE, "ezoracle.c")
_lock = threading.Lock()
_lib = None

MAXNU, MAXPROD = 8, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no -ffast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ezoracle.h"))
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrProblem(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int),
        ("A", ctypes.c_double * 9),
        ("lam", ctypes.c_double),
        ("r_real", ctypes.c_double),
        ("r_recip", ctypes.c_double),
        ("n_distinct", ctypes.c_int),
        ("nu", ctypes.c_double * MAXNU),
        ("n_prod", ctypes.c_int),
        ("expo", (ctypes.c_int * MAXNU) * MAXPROD),
        ("u_rule", ctypes.c_int),
        ("n_u", ctypes.c_int),
        ("n_v", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("ell", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_phi.restype = ctypes.c_double
            L.or_phi.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_expint_e1.restype = ctypes.c_double
            L.or_expint_e1.argtypes = [ctypes.c_double]
            L.or_gauss_legendre01.argtypes = [ctypes.c_int, dp, dp]
            L.or_hadamard.restype = ctypes.c_double
            L.or_hadamard.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.or_epstein_zeta.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp, dp]
            L.or_epstein_zeta_nd.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp, dp]
            L.or_epstein_zeta_reg.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, dp]
            L.or_s_hat.restype = ctypes.c_double
            L.or_s_hat.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            pp = ctypes.POINTER(OrProblem)
            L.or_n_sectors.argtypes = [pp]
            L.or_n_u_total.argtypes = [pp]
            L.or_u_rule.argtypes = [pp, dp, dp]
            L.or_nbody.argtypes = [pp, ctypes.c_int, dp, dp, dp]
            L.or_nbody_line.argtypes = [pp, ctypes.c_int, ctypes.c_int, dp]
            L.or_nbody_node.argtypes = [pp, ctypes.c_int, ctypes.c_double, dp, dp, dp]
            L.or_reg_taylor.argtypes = [pp, ctypes.c_int, dp, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(x, d=None) -> np.ndarray:
    a = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
    if d is not None and a.size < 3:
        a = np.concatenate([a, np.zeros(3 - a.size)])
    return a


def phi(a: float, t: float) -> float:
    """Phi_a(t) = t^{-a} Gamma(a, t)."""
    return lib().or_phi(float(a), float(t))


def e1(t: float) -> float:
    return lib().or_expint_e1(float(t))


def gauss_legendre01(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre01(n, _dp(x), _dp(w))
    return x, w


def hadamard(mu: float, m: int, eps: float, w2: float) -> float:
    return lib().or_hadamard(float(mu), int(m), float(eps), float(w2))


class OracleError(RuntimeError):
    pass


def epstein_zeta(A, nu, x, y, lam=1.0, r_real=8.0, r_recip=8.0) -> complex:
    """Z_{Lambda,nu}(x, y) (Def. "Epstein zeta function") by the incomplete-gamma splitting."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    d = A.shape[0]
    xv, yv = _vec(x, 3), _vec(y, 3)
    re, im = ctypes.c_double(), ctypes.c_double()
    rc = lib().or_epstein_zeta(d, _dp(A), float(nu), _dp(xv), _dp(yv), float(lam), float(r_real),
                               float(r_recip), ctypes.byref(re), ctypes.byref(im))
    if rc:
        raise OracleError(f"or_epstein_zeta rc={rc}")
    return complex(re.value, im.value)


def epstein_zeta_nd(A, nu, x, y, lam=1.0, r_real=8.0, r_recip=8.0) -> complex:
    """Z_{Lambda,nu}(x, y) for any dimension d <= 6 (A row-major d x d)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    d = A.shape[0]
    xv = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
    yv = np.ascontiguousarray(np.atleast_1d(np.asarray(y, dtype=np.float64)))
    if xv.size != d or yv.size != d:
        raise ValueError("x and y need d components")
    re, im = ctypes.c_double(), ctypes.c_double()
    rc = lib().or_epstein_zeta_nd(d, _dp(A.reshape(-1)), float(nu), _dp(xv), _dp(yv), float(lam), float(r_real),
                                  float(r_recip), ctypes.byref(re), ctypes.byref(im))
    if rc:
        raise OracleError(f"or_epstein_zeta_nd rc={rc}")
    return complex(re.value, im.value)


def epstein_zeta_reg(A, nu, k, lam=1.0, r_real=8.0, r_recip=8.0) -> float:
    A = np.ascontiguousarray(A, dtype=np.float64)
    kv = _vec(k, 3)
    out = ctypes.c_double()
    rc = lib().or_epstein_zeta_reg(A.shape[0], _dp(A), float(nu), _dp(kv), float(lam), float(r_real),
                                   float(r_recip), ctypes.byref(out))
    if rc:
        raise OracleError(f"or_epstein_zeta_reg rc={rc}")
    return out.value


def s_hat(d: int, nu: float, k) -> float:
    kv = _vec(k, 3)
    return lib().or_s_hat(int(d), float(nu), _dp(kv))


def make_problem(prob) -> OrProblem:
    """Convert a workloads.Problem into the C struct."""
    P = OrProblem()
    d = prob.A.shape[0]
    P.d = d
    A = np.zeros(9)
    A[: d * d] = np.asarray(prob.A, dtype=np.float64).reshape(-1)
    for i in range(9):
        P.A[i] = A[i]
    q = prob.quad
    P.lam, P.r_real, P.r_recip = q.lam, q.r_real, q.r_recip
    P.n_distinct = len(prob.nu)
    for j, v in enumerate(prob.nu):
        P.nu[j] = v
    P.n_prod = len(prob.expo)
    for p, row in enumerate(prob.expo):
        for j, e in enumerate(row):
            P.expo[p][j] = int(e)
    P.u_rule, P.n_u, P.n_v, P.eps, P.ell = q.u_rule, q.n_u, q.n_v, q.eps, q.ell
    return P


def n_sectors(prob) -> int:
    P = make_problem(prob)
    return lib().or_n_sectors(ctypes.byref(P))


def n_u_total(prob) -> int:
    P = make_problem(prob)
    return lib().or_n_u_total(ctypes.byref(P))


def u_rule(prob):
    P = make_problem(prob)
    n = lib().or_n_u_total(ctypes.byref(P))
    u, w = np.zeros(n), np.zeros(n)
    lib().or_u_rule(ctypes.byref(P), _dp(u), _dp(w))
    return u, w


def nbody(prob, threads: int = 1, lines: bool = False):
    """Lattice sums of every product of `prob` (Thm "Epstein representation" +
    Cor. "Duffy transformation"; eps-split near part for u_rule 2)."""
    P = make_problem(prob)
    L = lib()
    ns = L.or_n_sectors(ctypes.byref(P))
    nu_t = L.or_n_u_total(ctypes.byref(P))
    npr = P.n_prod
    out = np.zeros(npr)
    far = np.zeros(ns * nu_t * npr) if lines else None
    near = np.zeros(ns * npr) if lines else None
    rc = L.or_nbody(ctypes.byref(P), int(threads), _dp(out), _dp(far) if lines else None,
                    _dp(near) if lines else None)
    if rc:
        raise OracleError(f"or_nbody rc={rc}")
    if lines:
        return out, far.reshape(ns, nu_t, npr), near.reshape(ns, npr)
    return out


def nbody_line(prob, sector: int, iu: int) -> np.ndarray:
    P = make_problem(prob)
    out = np.zeros(P.n_prod)
    rc = lib().or_nbody_line(ctypes.byref(P), int(sector), int(iu), _dp(out))
    if rc:
        raise OracleError(f"or_nbody_line rc={rc}")
    return out


def nbody_node(prob, sector: int, u: float, v):
    P = make_problem(prob)
    vv = _vec(v if len(np.atleast_1d(v)) else [0.0], 3)
    f = np.zeros(P.n_prod)
    kt = np.zeros(3)
    rc = lib().or_nbody_node(ctypes.byref(P), int(sector), float(u), _dp(vv), _dp(f), _dp(kt))
    if rc:
        raise OracleError(f"or_nbody_node rc={rc}")
    return f, kt[: P.d]


def reg_taylor(prob, j: int, w) -> np.ndarray:
    P = make_problem(prob)
    wv = _vec(w, 3)
    C = np.zeros(P.ell + 1)
    rc = lib().or_reg_taylor(ctypes.byref(P), int(j), _dp(wv), _dp(C))
    if rc:
        raise OracleError(f"or_reg_taylor rc={rc}")
    return C


def atm_energy(parts) -> float:
    """Prop. (ATM): E = zeta(3,3,3)/24 - 3/16 zeta(-1,5,5) + 3/8 zeta(1,3,5)."""
    z333, zm155, z135 = parts
    return z333 / 24.0 - 3.0 * zm155 / 16.0 + 3.0 * z135 / 8.0
