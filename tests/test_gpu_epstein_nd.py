"""The Epstein zeta function in d = 4, 5, 6 (Sec. 6: the method in any dimension) on the GPU,
through the C ABI, against the oracle's d-dimensional splitting (FP64 form, 1e-13 relative with
an absolute floor of 1), and against closed forms that do not involve the oracle."""
import math

import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-13
RT = math.sqrt(45.0 / math.pi)  # the device's cutoff radius in units of lam (pi r^2 / lam^2 = 45)


@pytest.fixture(scope="module")
def ez():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_11989_gb300 import build, ezeta

    build.build()
    return ezeta


def _skew(d: int, seed: int) -> np.ndarray:
    A = np.eye(d) + 0.25 * np.random.default_rng(seed).uniform(-1.0, 1.0, (d, d))
    return A / abs(np.linalg.det(A)) ** (1.0 / d)


def _lattice(name: str) -> np.ndarray:
    return _skew(int(name[-1]), 5) if name.startswith("skew") else W.lattice(name)


ND_CASES = [("Z4", [-1.0, 1.0, 3.0, 4.0, 5.0, 9.0]), ("D4", [2.0, 3.5, 6.0]), ("skew4", [-2.5, 4.0, 7.25]),
            ("Z5", [3.0, 5.0, 6.5]), ("D5", [1.5, 7.0]), ("skew5", [4.5, 8.0]), ("Z6", [2.0, 6.0, 8.0]),
            ("E6", [3.0, 7.5]), ("skew6", [5.0, 9.0])]


@pytest.mark.parametrize("lat,nus", ND_CASES, ids=[c[0] for c in ND_CASES])
def test_epstein_zeta_nd_parity(ez, oracle_mod, lat, nus):
    import torch

    A = _lattice(lat)
    d = A.shape[0]
    L = ez.Lattice(A)
    rng = np.random.default_rng(31 + d)
    Binv = np.linalg.inv(A).T
    ys = np.concatenate([rng.uniform(-0.5, 0.5, (24, d)) @ Binv.T, rng.uniform(-2, 2, (4, d))])
    xs = [np.zeros(d), A @ rng.uniform(-0.5, 0.5, d), A @ np.ones(d)]
    lam = abs(np.linalg.det(A)) ** (1.0 / d)
    for nu in nus:
        for x in xs:
            re, im = ez.ez_epstein_zeta(L, nu, x, ys)
            yt = torch.tensor(ys, dtype=torch.float64, device="cuda")
            re2, im2 = ez.ez_epstein_zeta(L, nu, x, yt)
            assert np.array_equal(re, re2.cpu().numpy()) and np.array_equal(im, im2.cpu().numpy())
            for i in range(0, len(ys), 2):
                z = oracle_mod.epstein_zeta_nd(A, nu, x, ys[i], lam, 1.1 * RT * lam, 1.1 * RT / lam)
                assert abs(complex(re[i], im[i]) - z) <= TOL * max(1.0, abs(z)), (lat, nu, x, i, re[i], im[i], z)


@pytest.mark.parametrize("s", [2.5, 3.0, 4.5])
def test_z4_four_squares_closed_form(ez, s):
    # Jacobi: the number of representations of n as a sum of four squares is 8 sigma(n) for odd
    # n and 24 sigma(odd part of n) for even n, so sum' |m|^{-2s} over Z^4 = 8 (1 - 4^{1-s})
    # zeta(s) zeta(s - 1) (s > 2); mpmath gives the zeta values
    mpmath = pytest.importorskip("mpmath")
    ref = float(8 * (1 - mpmath.mpf(4) ** (1 - s)) * mpmath.zeta(s) * mpmath.zeta(s - 1))
    L = ez.Lattice(np.eye(4))
    re, im = ez.ez_epstein_zeta(L, 2 * s, np.zeros(4), np.zeros((1, 4)))
    assert re[0] == pytest.approx(ref, rel=TOL) and abs(im[0]) < TOL * ref


def test_nd_quasi_periodicity_and_poles(ez):
    # Z(x, y + g*) = Z(x, y) for g* in the dual lattice; Z(x + z, y) = e^{-2 pi i y.z} Z(x, y)
    # for z in the lattice; y in the dual lattice with nu <= d is a pole (EZ_EDOMAIN)
    A = W.lattice("D5")
    d = 5
    L = ez.Lattice(A)
    rng = np.random.default_rng(3)
    x = A @ rng.uniform(-0.5, 0.5, d)
    y = np.linalg.inv(A).T @ rng.uniform(-0.5, 0.5, d)
    g = np.linalg.inv(A).T @ np.array([1.0, -2.0, 0.0, 1.0, 3.0])
    z = A @ np.array([2.0, 0.0, -1.0, 1.0, 1.0])
    nu = 6.3
    re, im = ez.ez_epstein_zeta(L, nu, x, np.stack([y, y + g]))
    a, b = complex(re[0], im[0]), complex(re[1], im[1])
    assert abs(a - b) <= 1e-13 * abs(a)
    re2, im2 = ez.ez_epstein_zeta(L, nu, x + z, y[None, :])
    c = complex(re2[0], im2[0])
    assert abs(c - np.exp(-2j * np.pi * (y @ z)) * a) <= 1e-13 * abs(a)
    # (y = 0, and an integer y on Z^5, whose reduction is exact)
    with pytest.raises(ez.EzError) as e:
        ez.ez_epstein_zeta(L, 4.0, np.zeros(d), np.zeros((1, d)))
    assert e.value.code == ez.EZ_EDOMAIN
    with pytest.raises(ez.EzError) as e:
        ez.ez_epstein_zeta(ez.Lattice(np.eye(5)), 5.0, x, np.array([[0.3, 0.1, 0, 0, 0], [1.0, 0, -2.0, 0, 1.0]]))
    assert e.value.code == ez.EZ_EDOMAIN
    # nu > d at y = 0 is finite: the g* = 0 term is the limit -1/a of Phi_a(t) - Gamma(a) t^{-a}
    re, _ = ez.ez_epstein_zeta(L, 7.0, np.zeros(d), np.zeros((1, d)))
    assert np.isfinite(re[0]) and re[0] > 0.0


def test_lattice_sums_refuse_d_above_3(ez):
    # the Duffy nodes, near part and static scratch are built for d <= 3: EZ_EUNSUPPORTED
    import torch

    L = ez.Lattice(W.lattice("D4"))
    q = ez.quadrature(W.Quad(n_u=4, n_v=4))
    for call in (lambda: ez.ez_lattice_sum_nbody(L, [5.0, 5.0], q), lambda: ez.ez_atm_energy(L, q)):
        with pytest.raises(ez.EzError) as e:
            call()
        assert e.value.code == ez.EZ_EUNSUPPORTED
    y = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    re = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(ez.EzError) as e:
        ez.ez_epstein_zeta_static(L, 5.0, np.zeros(4), y, re)
    assert e.value.code == ez.EZ_EUNSUPPORTED
