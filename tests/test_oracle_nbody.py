"""Pins of the oracle's n-body lattice sums: Thm "Epstein representation", Cor.
"Duffy transformation", and the eps-split meromorphic continuation of Sec. 3.

References: the exact d=1 value of zeta^(3)(4,4,4) from the Bernoulli closed form of
Z_4 (rational times pi^12), Cor. "one- and two-body" (zeta^(1) = 0, zeta^(2)(nu1,nu2)
= Z_{nu1+nu2}(0)), brute-force sums of Def. "Many-body zeta function" for large
exponents (the paper's own test, Sec. 4.3/4.4), the ATM values printed in Sec. 4.3,
invariance under the splitting parameter, the scaling law and the bound of Sec. 4.4.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W
from tests import brute

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def exact_zeta3_Z_444():
    # Z_{Z,4}(k) = -(2 pi)^4 B_4(k) / 24 on [0,1]; zeta^(3) = 2 int_0^{1/2} Z_4(k)^3 dk
    b = [Fraction(-1, 30), Fraction(0), Fraction(1), Fraction(-2), Fraction(1)]
    c = [Fraction(0)] * 13
    for i, x in enumerate(b):
        for j, y in enumerate(b):
            for k, z in enumerate(b):
                c[i + j + k] += x * y * z
    I = sum(ci * Fraction(1, 2) ** (i + 1) / (i + 1) for i, ci in enumerate(c))
    return 2.0 * (-(2 * math.pi) ** 4 / 24) ** 3 * float(I)


@pytest.mark.parametrize("n_u", [7, 64, 4096])
def test_config1_exact(oracle_mod, n_u):
    p = W.nbody_problem("Z", 4.0, 3, W.config1(n_u))
    assert oracle_mod.nbody(p, threads=4)[0] == pytest.approx(exact_zeta3_Z_444(), rel=1e-14)


@pytest.mark.parametrize("lat,nu", [("Z", 4.0), ("Z", 3.0), ("square", 3.0), ("hexagonal", 3.0), ("hexagonal", 4.0), ("fcc", 6.0), ("bcc", 5.0)])
def test_one_and_two_body(oracle_mod, lat, nu):
    d = W.DIM_OF[lat]
    q = W.Quad(n_u=20, n_v=14 if d == 3 else 24, u_rule=2 if (nu - d) % 2 == 0 else 1, lam=1.0, r_real=6.0, r_recip=6.0)
    p1 = W.nbody_problem(lat, nu, 1, q)
    assert abs(oracle_mod.nbody(p1, threads=8)[0]) < 1e-13
    p2 = W.nbody_problem(lat, nu, 2, q)
    ref = oracle_mod.epstein_zeta(p2.A, 2 * nu, np.zeros(d), np.zeros(d), 1.0, 8, 8).real
    assert oracle_mod.nbody(p2, threads=8)[0] == pytest.approx(ref, rel=1e-13)


def test_d1_three_body_vs_direct(oracle_mod):
    nus = (6.0, 7.0, 8.0)
    prob = W.Problem("z", W.lattice("Z"), list(nus), [[1, 1, 1]], W.Quad(n_u=8, n_v=1, u_rule=2, lam=1.0, r_real=9, r_recip=9))
    got = oracle_mod.nbody(prob)[0]
    ref = brute.zeta_n_direct(W.lattice("Z"), nus, 600)
    assert got == pytest.approx(ref, rel=2e-14)


def test_d2_three_body_vs_direct(oracle_mod):
    A = W.lattice("hexagonal", unit_density=False)
    nus = (12.0, 13.0, 14.0)
    prob = W.Problem("z", A, list(nus), [[1, 1, 1]], W.Quad(n_u=24, n_v=20, u_rule=2, lam=1.0, r_real=7, r_recip=7))
    got = oracle_mod.nbody(prob, threads=8)[0]
    ref = brute.zeta_n_direct(A, nus, 14)
    assert got == pytest.approx(ref, rel=1e-13)


def test_hex_four_body_vs_direct(oracle_mod):
    # Sec. 4.4: four-body zeta on the hexagonal lattice at large nu against direct sums
    A = W.lattice("hexagonal", unit_density=False)
    nu = 14.0
    prob = W.nbody_problem("hexagonal", nu, 4, W.Quad(n_u=24, n_v=20, u_rule=2, lam=1.0, r_real=7, r_recip=7))
    prob.A = A
    got = oracle_mod.nbody(prob, threads=8)[0]
    ref = brute.zeta_n_direct(A, (nu,) * 4, 5)
    assert got == pytest.approx(ref, rel=1e-13)


def test_fcc_three_body_vs_direct(oracle_mod):
    A = W.lattice("fcc", unit_density=False)
    nus = (16.0, 16.0, 16.0)
    prob = W.Problem("z", A, list(nus), [[3]], W.Quad(n_u=16, n_v=12, u_rule=2, lam=1.0, r_real=6, r_recip=6))
    got = oracle_mod.nbody(prob, threads=8)[0]
    ref = brute.zeta_n_direct(A, nus, 5)
    assert got == pytest.approx(ref, rel=1e-12)


def test_atm_d1_printed_value(oracle_mod):
    p = W.atm_problem("Z", W.Quad(n_u=12, n_v=1, u_rule=2, eps=1e-2, ell=4, lam=1.0, r_real=8, r_recip=8))
    E = oracle_mod.atm_energy(oracle_mod.nbody(p))
    assert E == pytest.approx(GOLD["atm_Z_method"]["value"], abs=3e-14)
    assert E == pytest.approx(GOLD["atm_Z_direct_L5000"]["value"], abs=3e-14)


def test_atm_d1_vs_direct_sum_of_definition(oracle_mod):
    # Def. "ATM": E = 1/6 sum' U(x, y), brute force on L = 400 (tail ~ 1e-9 at L=400)
    p = W.atm_problem("Z", W.Quad(n_u=12, n_v=1, u_rule=2, lam=1.0, r_real=8, r_recip=8))
    E = oracle_mod.atm_energy(oracle_mod.nbody(p))
    assert E == pytest.approx(brute.atm_direct(W.lattice("Z"), 400), abs=1e-8)


def test_atm_square_printed_value(oracle_mod):
    p = W.atm_problem("square", W.Quad(n_u=12, n_v=20, u_rule=2, eps=1e-2, ell=4, lam=1.0, r_real=6, r_recip=6))
    E = oracle_mod.atm_energy(oracle_mod.nbody(p, threads=8))
    assert E == pytest.approx(GOLD["atm_square_method"]["value"], abs=1.5e-13)
    assert E == pytest.approx(GOLD["atm_square_direct_L1600"]["value"], abs=5e-13)


@pytest.mark.parametrize("lat", ["square", "hexagonal"])
def test_taylor_order_error_decay(oracle_mod, lat):
    # Table "taylor": error of zeta^(3)(1,3,5), (-1,5,5) vs ell (reference ell=6), eps=1e-2
    def parts(ell):
        q = W.Quad(n_u=10, n_v=14, u_rule=2, eps=1e-2, ell=ell, lam=1.0, r_real=6, r_recip=6)
        return oracle_mod.nbody(W.atm_problem(lat, q), threads=8)

    ref = parts(6)
    errs = {ell: np.abs(parts(ell) - ref) / np.abs(ref) for ell in (0, 1, 2, 3)}
    key = "square" if lat == "square" else "hex"
    tab_135 = GOLD["taylor_error_ell"][f"{key}_135"]
    tab_m155 = GOLD["taylor_error_ell"][f"{key}_m155"]
    for ell in (0, 1, 2):
        for got, printed in ((errs[ell][2], tab_135[ell]), (errs[ell][1], tab_m155[ell])):
            assert 0.8 * printed < got < 1.25 * printed, (ell, got, printed)
    assert errs[3][2] < 1e-15 and errs[3][1] < 5e-15


def test_lambda_invariance_atm_d2(oracle_mod):
    vals = []
    for lam in (0.9, 1.0, 1.25):
        q = W.Quad(n_u=10, n_v=14, u_rule=2, lam=lam, r_real=7.5, r_recip=7.5)
        vals.append(oracle_mod.nbody(W.atm_problem("hexagonal", q), threads=8))
    for v in vals[1:]:
        np.testing.assert_allclose(v, vals[0], rtol=1e-13)


def test_scaling_law_and_bound(oracle_mod):
    q = W.Quad(n_u=16, n_v=16, u_rule=1, lam=1.0, r_real=6, r_recip=6)
    base = W.nbody_problem("hexagonal", 3.0, 3, q)
    v0 = oracle_mod.nbody(base, threads=8)[0]
    s = 1.17
    scaled = W.nbody_problem("hexagonal", 3.0, 3, W.Quad(n_u=16, n_v=16, u_rule=1, lam=s, r_real=6 * s, r_recip=6 / s), scale=s)
    assert oracle_mod.nbody(scaled, threads=8)[0] == pytest.approx(v0 * s**-9, rel=1e-13)
    z3 = oracle_mod.epstein_zeta(base.A, 3.0, [0, 0], [0, 0], 1.0, 8, 8).real
    assert 0 < v0 <= z3**3


def test_duffy_sector_count_and_weights(oracle_mod):
    for lat, ns in (("Z", 1), ("square", 4), ("fcc", 12)):
        p = W.nbody_problem(lat, 6.0, 1, W.Quad(n_u=4, n_v=4))
        assert oracle_mod.n_sectors(p) == ns
    # the weights of the Duffy rule integrate the constant 1 over the half BZ:
    # V int_BZ 1 dk = 1 -> a "product" of zero factors sums to 1
    p = W.Problem("one", W.lattice("bcc"), [6.0], [[0]], W.Quad(n_u=8, n_v=6, u_rule=1))
    assert oracle_mod.nbody(p)[0] == pytest.approx(1.0, rel=1e-14)
