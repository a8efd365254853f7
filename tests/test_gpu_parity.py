"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerance: the plain FP64 form must match the oracle to 1e-13 relative (the
target stated for this path); line partial sums are compared element by element
with an absolute floor of 1e-13 times the largest line of the same request.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(scope="module")
def ez():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_11989_gb300 import build, ezeta

    build.build()
    return ezeta


def _close(got, ref, tol=TOL, floor=0.0):
    got, ref = np.asarray(got), np.asarray(ref)
    return np.all(np.abs(got - ref) <= tol * np.maximum(np.abs(ref), floor))


# ------------------------------------------------------------------ Epstein zeta
CASES = [("Z", [-1, 1, 2, 3, 4, 9]), ("square", [-1, 1, 2, 3, 5, 6]), ("hexagonal", [-3, -1, 1, 3, 4, 7]),
         ("kappa=2", [1, 3]), ("sc", [-1, 1, 3, 4, 6]), ("fcc", [-1, 1, 2, 3, 5, 6, 9, 12]), ("bcc", [-1, 3, 5])]


@pytest.mark.parametrize("lat,nus", CASES)
def test_epstein_zeta_parity(ez, oracle_mod, lat, nus):
    import torch

    A = W.lattice(lat)
    d = A.shape[0]
    L = ez.Lattice(A)
    rng = np.random.default_rng(17)
    Binv = np.linalg.inv(A).T
    ys = np.concatenate([rng.uniform(-0.5, 0.5, (40, d)) @ Binv.T, rng.uniform(-3, 3, (8, d))])
    xs = [np.zeros(d), A @ rng.uniform(-0.5, 0.5, d), A @ np.ones(d)]
    for nu in nus:
        for x in xs:
            re, im = ez.ez_epstein_zeta(L, nu, x, ys)
            # device-resident input/output too
            yt = torch.tensor(ys, dtype=torch.float64, device="cuda")
            re2, im2 = ez.ez_epstein_zeta(L, nu, x, yt)
            assert np.array_equal(re, re2.cpu().numpy()) and np.array_equal(im, im2.cpu().numpy())
            lam = abs(np.linalg.det(A)) ** (1.0 / d)
            for i in range(0, len(ys), 3):
                z = oracle_mod.epstein_zeta(A, nu, x, ys[i], lam, 9.0 * lam, 9.0 / lam)
                scale = max(1.0, abs(z))
                assert abs(complex(re[i], im[i]) - z) <= TOL * scale, (lat, nu, x, i, re[i], im[i], z)


def test_epstein_zeta_edge_cases(ez, oracle_mod):
    L = ez.Lattice(W.lattice("square"))
    # m = 0 is a no-op
    re, im = ez.ez_epstein_zeta(L, 3.0, [0, 0], np.zeros((0, 2)))
    assert re.size == 0
    # y in the reciprocal lattice with nu <= d is a pole
    with pytest.raises(ez.EzError) as e:
        ez.ez_epstein_zeta(L, 1.0, [0, 0], np.array([[0.0, 0.0], [0.1, 0.2]]))
    assert e.value.code == ez.EZ_EDOMAIN
    # ... but nu > d at y = 0 is Z(0)
    re, _ = ez.ez_epstein_zeta(L, 5.0, [0, 0], np.zeros((1, 2)))
    assert _close(re[0], oracle_mod.epstein_zeta(np.eye(2), 5.0, [0, 0], [0, 0], 1.0, 8, 8).real)
    for bad_nu, code in ((-2.0, ez.EZ_EDOMAIN), (0.0, ez.EZ_EDOMAIN), (float("nan"), ez.EZ_EINVAL)):
        with pytest.raises(ez.EzError) as e:
            ez.ez_epstein_zeta(L, bad_nu, [0, 0], np.zeros((1, 2)))
        assert e.value.code == code
    with pytest.raises(ez.EzError) as e:
        ez.Lattice(np.array([[1.0, 2.0], [2.0, 4.0]]))
    assert e.value.code == ez.EZ_EINVAL


# ------------------------------------------------------------------ lattice sums
def _run(ez, prob):
    L = ez.Lattice(prob.A)
    spec = ez.sum_spec(prob.nu, prob.expo)
    q = ez.quadrature(prob.quad)
    out, lines, offs = ez.ez_lattice_sums([L], [spec], [q], lines=True)
    return out[0, : len(prob.expo)], lines[offs[0]: offs[1], : len(prob.expo)]


def _compare_with_oracle(ez, oracle_mod, prob, threads=16):
    got, lines = _run(ez, prob)
    ref, far, near = oracle_mod.nbody(prob, threads=threads, lines=True)
    ns, nu_t, npr = far.shape
    ref_lines = far.reshape(ns * nu_t, npr)
    if prob.quad.u_rule == 2:
        ref_lines = np.concatenate([ref_lines, near])
    assert lines.shape == ref_lines.shape
    floor = np.max(np.abs(ref_lines), axis=0)
    assert np.all(np.abs(lines - ref_lines) <= TOL * np.maximum(np.abs(ref_lines), floor)), prob.name
    assert _close(got, ref), (prob.name, got, ref)
    return got, ref


SMALL = [
    W.nbody_problem("Z", 4.0, 3, W.config1(64)),
    W.nbody_problem("Z", 4.0, 3, W.config1(300)),  # ragged d=1 block tail
    W.nbody_problem("square", 3.0, 3, W.config2(32)),
    W.nbody_problem("hexagonal", 3.0, 3, W.config2(34)),
    W.nbody_problem("hexagonal", 3.0, 5, W.Quad(n_u=10, n_v=140, lam=1.3, r_real=7, r_recip=5)),  # n_v > 128
    W.nbody_problem("fcc", 6.0, 3, W.Quad(n_u=5, n_v=19, lam=1.0, r_real=4.5, r_recip=4.5)),  # ragged v2 chunk
    W.nbody_problem("bcc", 5.0, 2, W.Quad(n_u=3, n_v=8, u_rule=2, lam=1.0, r_real=4.5, r_recip=4.5)),  # log case
    W.atm_problem("Z", W.Quad(n_u=12, n_v=1, u_rule=2, lam=1.0, r_real=8, r_recip=8)),
    W.atm_problem("square", W.Quad(n_u=6, n_v=10, u_rule=2, lam=1.0, r_real=6, r_recip=6)),
    W.atm_problem("hexagonal", W.Quad(n_u=6, n_v=9, u_rule=2, lam=1.2, r_real=6, r_recip=6)),
    W.atm_problem("fcc", W.Quad(n_u=3, n_v=6, u_rule=2, lam=1.0, r_real=4.5, r_recip=4.5)),
    W.atm_problem("sc", W.Quad(n_u=3, n_v=5, u_rule=2, lam=1.0, r_real=4.5, r_recip=4.5)),
]


@pytest.mark.parametrize("prob", SMALL, ids=[p.name + f"-{i}" for i, p in enumerate(SMALL)])
def test_nbody_parity_small(ez, oracle_mod, prob):
    _compare_with_oracle(ez, oracle_mod, prob)


def test_config1_full_size(ez, oracle_mod):
    prob = W.nbody_problem("Z", 4.0, 3, W.config1(4096))
    got, ref = _compare_with_oracle(ez, oracle_mod, prob)
    # and the closed form of the paper's 1-D case (Bernoulli), see the oracle pins
    assert got[0] == pytest.approx(0.38504407962833566, rel=1e-14)


@pytest.mark.parametrize("lat", ["square", "hexagonal"])
def test_config2_full_size(ez, oracle_mod, lat):
    prob = W.nbody_problem(lat, 3.0, 3, W.config2(256))
    _compare_with_oracle(ez, oracle_mod, prob)


def test_config3_atm_full_size_sampled_lines(ez, oracle_mod):
    # full size (12 sectors x 48 u x 64^2 v): 32 sampled far lines (every sector at least
    # twice) and the near-part line of every sector against the oracle
    prob = W.atm_problem("fcc", W.config3())
    got, lines = _run(ez, prob)
    ns, nu_t = oracle_mod.n_sectors(prob), oracle_mod.n_u_total(prob)
    rng = np.random.default_rng(5)
    picks = [(s % ns, int(rng.integers(nu_t))) for s in range(32)] + [(s, -1) for s in range(ns)]
    with ThreadPoolExecutor(16) as ex:
        refs = list(ex.map(lambda si: oracle_mod.nbody_line(prob, si[0], si[1]), picks))
    floor = np.max(np.abs(lines), axis=0)
    for (s, iu), ref in zip(picks, refs):
        row = lines[s * nu_t + iu] if iu >= 0 else lines[ns * nu_t + s]
        assert np.all(np.abs(row - ref) <= TOL * np.maximum(np.abs(ref), floor[: len(ref)])), (s, iu, row, ref)
    # the lines add up to the value (fixed-order compensated reduction): against the exactly
    # rounded sum of the lines, relative to the sum of their magnitudes (the lines cancel)
    exact = np.array([math.fsum(lines[:, q]) for q in range(lines.shape[1])])
    assert np.all(np.abs(got - exact) <= 1e-14 * np.sum(np.abs(lines), axis=0))


def _sampled_lines(ez, oracle_mod, prob, seed, n_pick, tol, prec=None):
    """Full-size sum on the GPU; a few of its quadrature lines from the oracle (run at the
    explicit splitting parameter when the GPU sum uses the default one)."""
    L = ez.Lattice(prob.A)
    q = ez.quadrature(prob.quad) if prec is None else ez.quadrature(prob.quad, prec=prec)
    out, lines, offs = ez.ez_lattice_sums([L], [ez.sum_spec(prob.nu, prob.expo)], [q], lines=True)
    npr = len(prob.expo)
    got, lines = out[0, :npr], lines[offs[0]: offs[1], :npr]
    ref_prob = W.explicit_splitting(prob)
    ns, nu_t = oracle_mod.n_sectors(ref_prob), oracle_mod.n_u_total(ref_prob)
    rng = np.random.default_rng(seed)
    picks = [(int(rng.integers(ns)), int(rng.integers(nu_t))) for _ in range(n_pick)]
    if prob.quad.u_rule == 2:
        picks.append((int(rng.integers(ns)), -1))
    with ThreadPoolExecutor(8) as ex:
        refs = list(ex.map(lambda si: oracle_mod.nbody_line(ref_prob, si[0], si[1]), picks))
    floor = np.max(np.abs(lines), axis=0)
    for (s, iu), ref in zip(picks, refs):
        row = lines[s * nu_t + iu] if iu >= 0 else lines[ns * nu_t + s]
        assert np.all(np.abs(row - ref) <= tol * np.maximum(np.abs(ref), floor[: len(ref)])), (s, iu, row, ref)
    # the lines add up to the value (fixed-order compensated reduction; the numpy sum of
    # lines of both signs is only accurate relative to the sum of their magnitudes)
    assert np.all(np.abs(got - lines.sum(axis=0)) <= 1e-14 * np.sum(np.abs(lines), axis=0))
    return got


@pytest.mark.parametrize("n", [3, 8])
def test_config4_full_size_sampled_lines(ez, oracle_mod, n):
    """fcc, nu = 6, 12 sectors x 32 u x 48^2 v nodes, default splitting parameter."""
    prob = W.nbody_problem("fcc", 6.0, n, W.Quad(n_u=32, n_v=48, lam=0.0, r_real=0.0, r_recip=0.0))
    _sampled_lines(ez, oracle_mod, prob, 40 + n, 5, TOL)


@pytest.mark.parametrize("lat", ["sc", "bcc"])
def test_config3_atm_default_lambda_sampled_lines(ez, oracle_mod, lat):
    prob = W.atm_problem(lat, W.Quad(n_u=8, n_v=64, u_rule=2, lam=0.0, r_real=0.0, r_recip=0.0))
    _sampled_lines(ez, oracle_mod, prob, 7, 4, TOL)


AUTO = dict(lam=0.0, r_real=0.0, r_recip=0.0)


@pytest.mark.parametrize("prob", [
    W.nbody_problem("Z", 4.0, 3, W.Quad(n_u=64, n_v=1, **AUTO), scale=1.2),
    W.nbody_problem("hexagonal", 3.0, 3, W.Quad(n_u=16, n_v=16, **AUTO), scale=0.9),
    W.atm_problem("square", W.Quad(n_u=6, n_v=10, u_rule=2, **AUTO), scale=1.1),
    W.nbody_problem("fcc", 6.0, 4, W.Quad(n_u=4, n_v=11, **AUTO), scale=1.3),
    W.atm_problem("bcc", W.Quad(n_u=3, n_v=6, u_rule=2, **AUTO)),
], ids=lambda p: p.name)
def test_default_splitting_parameter_matches_oracle(ez, oracle_mod, prob):
    """lam = 0 lets the library pick lam and the cutoffs; every quadrature line must agree
    with the oracle run at its own explicit lam = V^{1/d} (the sum does not depend on lam)."""
    got, lines = _run(ez, prob)
    ref, far, near = oracle_mod.nbody(W.explicit_splitting(prob), threads=16, lines=True)
    ref_lines = far.reshape(-1, far.shape[2])
    if prob.quad.u_rule == 2:
        ref_lines = np.concatenate([ref_lines, near])
    floor = np.max(np.abs(ref_lines), axis=0)
    assert np.all(np.abs(lines - ref_lines) <= TOL * np.maximum(np.abs(ref_lines), floor)), prob.name
    assert _close(got, ref), (prob.name, got, ref)


@pytest.mark.parametrize("prob,prec", [
    (W.nbody_problem("Z", 4.0, 3, W.config1(300)), 0),
    (W.nbody_problem("hexagonal", 3.0, 3, W.config2(34)), 0),
    (W.atm_problem("square", W.Quad(n_u=6, n_v=10, u_rule=2, lam=1.0, r_real=6, r_recip=6)), 0),
    (W.nbody_problem("fcc", 6.0, 3, W.Quad(n_u=5, n_v=19, **AUTO)), 0),
    (W.atm_problem("sc", W.Quad(n_u=3, n_v=12, u_rule=2, **AUTO)), 1),
], ids=["d1", "d2", "d2-atm-near", "d3", "d3-atm-mixed"])
def test_parts_add_up_to_the_whole(ez, prob, prec):
    """n_parts = 3 splits a sum over contiguous ranges of Duffy lines (near part in part
    0): each part's lines equal the whole sum's lines bitwise on its range and are zero
    elsewhere, and the three values add up to the whole value."""
    L = ez.Lattice(prob.A)
    spec = ez.sum_spec(prob.nu, prob.expo)
    npr = len(prob.expo)
    whole, wl, offs = ez.ez_lattice_sums([L], [spec], [ez.quadrature(prob.quad, prec=prec)], lines=True)
    wl = wl[offs[0]: offs[1], :npr]
    parts = [ez.quadrature(prob.quad, prec=prec, part=k, n_parts=3) for k in range(3)]
    vals, pl, poffs = ez.ez_lattice_sums([L] * 3, [spec] * 3, parts, lines=True)
    covered = np.zeros(len(wl), dtype=int)
    for k in range(3):
        lk = pl[poffs[k]: poffs[k + 1], :npr]
        nz = np.any(lk != 0.0, axis=1)
        assert np.array_equal(lk[nz], wl[nz])
        covered += nz
    assert np.all(covered[np.any(wl != 0.0, axis=1)] == 1)  # every line in exactly one part
    tot = vals[:, :npr].sum(axis=0)
    assert np.all(np.abs(tot - whole[0, :npr]) <= 1e-14 * np.sum(np.abs(wl), axis=0))


def test_nbody_api_matches_batch_and_is_deterministic(ez, oracle_mod):
    prob = W.nbody_problem("hexagonal", 3.0, 4, W.config2(40))
    L = ez.Lattice(prob.A)
    q = ez.quadrature(prob.quad)
    a = ez.ez_lattice_sum_nbody(L, [3.0] * 4, q)
    b = ez.ez_lattice_sum_nbody(L, [3.0] * 4, q)
    assert a == b
    many = ez.ez_lattice_sums([L, L, ez.Lattice(W.lattice("square"))],
                              [ez.sum_spec([3.0], [[4]])] * 3, [q] * 3)
    assert many[0, 0] == a and many[1, 0] == a
    q0 = ez.quadrature(prob.quad, dedupe=0)
    c = ez.ez_lattice_sum_nbody(L, [3.0] * 4, q0)  # one evaluation per factor
    assert _close(c, a, tol=1e-14)
    assert _close(a, oracle_mod.nbody(prob, threads=16)[0])


def test_atm_energy_api(ez, oracle_mod):
    import json
    import os

    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    for lat, key, tol in (("Z", "atm_Z_method", 3e-14), ("square", "atm_square_method", 1.5e-13)):
        q = W.Quad(n_u=12, n_v=1 if lat == "Z" else 20, u_rule=2, lam=1.0, r_real=8 if lat == "Z" else 6,
                   r_recip=8 if lat == "Z" else 6)
        E, parts = ez.ez_atm_energy(ez.Lattice(W.lattice(lat)), ez.quadrature(q))
        assert E == pytest.approx(gold[key]["value"], abs=tol)
        ref = oracle_mod.nbody(W.atm_problem(lat, q), threads=16)
        assert _close(parts, ref)


def test_sum_errors(ez):
    L = ez.Lattice(W.lattice("square"))
    q = ez.quadrature(W.config2(16))
    with pytest.raises(ez.EzError) as e:
        ez.ez_lattice_sum_nbody(L, [float("inf"), 3.0], q)
    assert e.value.code == ez.EZ_EINVAL
    with pytest.raises(ez.EzError) as e:  # d = 2, nu = (1, 1): mu = 2 + 2 (1 - 2) = 0
        ez.ez_lattice_sum_nbody(L, [1.0, 1.0], ez.quadrature(W.config2(16), u_rule=2))
    assert e.value.code == ez.EZ_EDOMAIN
    with pytest.raises(ez.EzError) as e:
        ez.ez_lattice_sum_nbody(L, [-2.0, 3.0], q)
    assert e.value.code == ez.EZ_EDOMAIN
    with pytest.raises(ez.EzError) as e:
        ez.ez_lattice_sum_nbody(L, [3.0], ez.quadrature(W.config2(16), n_u=0))
    assert e.value.code == ez.EZ_EINVAL


def test_mixed_batch_equals_single_requests(ez, oracle_mod):
    """A batch mixing d = 1, 2, 3, far-only and eps-split sums gives every sum exactly
    its single-request value (requests are independent inside a launch)."""
    probs = [
        W.nbody_problem("hexagonal", 3.0, 4, W.config2(24)),
        W.atm_problem("Z", W.Quad(n_u=8, n_v=1, u_rule=2, lam=1.0, r_real=8, r_recip=8)),
        W.atm_problem("fcc", W.Quad(n_u=2, n_v=6, u_rule=2, lam=1.0, r_real=4.5, r_recip=4.5)),
        W.nbody_problem("Z", 6.0, 2, W.config1(200)),
        W.nbody_problem("square", 4.0, 2, W.Quad(n_u=5, n_v=12, u_rule=2, lam=1.1, r_real=6, r_recip=5)),
        W.nbody_problem("bcc", 6.0, 3, W.Quad(n_u=4, n_v=17, lam=1.0, r_real=4.5, r_recip=4.5)),
    ]
    lats = [ez.Lattice(p.A) for p in probs]
    specs = [ez.sum_spec(p.nu, p.expo) for p in probs]
    quads = [ez.quadrature(p.quad) for p in probs]
    many, lines, offs = ez.ez_lattice_sums(lats, specs, quads, lines=True)
    b = ez.Batch(lats, specs, quads)
    # the batch fills its Phi tables on the first run and keeps them; the per-line sums are
    # written on request from the last run's segments: every run and its lines agree bitwise
    # with the one-shot path, which builds everything per call
    for _ in range(3):
        again = b.run()
        assert np.array_equal(again, many)
    blines, boffs = b.lines()
    assert np.array_equal(blines, lines) and list(boffs) == list(offs)
    for i, p in enumerate(probs):
        one, one_lines, one_offs = ez.ez_lattice_sums([lats[i]], [specs[i]], [quads[i]], lines=True)
        assert np.array_equal(one[0], many[i]), (i, one[0], many[i])
        assert np.array_equal(one_lines, lines[offs[i]: offs[i + 1]])
    # and against the oracle
    for i, p in enumerate(probs):
        ref = oracle_mod.nbody(p, threads=16)
        assert _close(many[i, : len(ref)], ref), (p.name, many[i], ref)


# ------------------------------------------------------------------ mixed form
MIXED_TOL = 1e-10  # stated bound of the mixed form (binary32 tails, binary64 heads)


def _compare_mixed(ez, oracle_mod, prob, threads=16):
    L = ez.Lattice(prob.A)
    spec = ez.sum_spec(prob.nu, prob.expo)
    npr = len(prob.expo)
    qm = ez.quadrature(prob.quad, prec=ez.EZ_MIXED)
    got, lines, offs = ez.ez_lattice_sums([L], [spec], [qm], lines=True)
    ref, far, near = oracle_mod.nbody(prob, threads=threads, lines=True)
    ref_lines = far.reshape(-1, npr)
    if prob.quad.u_rule == 2:
        ref_lines = np.concatenate([ref_lines, near])
    lines = lines[offs[0]: offs[1], :npr]
    floor = np.max(np.abs(ref_lines), axis=0)
    assert np.all(np.abs(lines - ref_lines) <= MIXED_TOL * np.maximum(np.abs(ref_lines), floor)), prob.name
    assert _close(got[0, :npr], ref, tol=MIXED_TOL), (prob.name, got[0, :npr], ref)
    return got[0, :npr], ref


@pytest.mark.parametrize("prob", SMALL, ids=[p.name + f"-{i}" for i, p in enumerate(SMALL)])
def test_mixed_parity_small(ez, oracle_mod, prob):
    _compare_mixed(ez, oracle_mod, prob)


@pytest.mark.parametrize("lat", ["square", "hexagonal"])
def test_mixed_config2_full_size_uses_binary32_tails(ez, oracle_mod, lat):
    prob = W.nbody_problem(lat, 3.0, 3, W.config2(256))
    got, ref = _compare_mixed(ez, oracle_mod, prob)
    L = ez.Lattice(prob.A)
    fp64 = ez.ez_lattice_sum_nbody(L, [3.0] * 3, ez.quadrature(prob.quad))
    assert fp64 != got[0]  # the tail really ran in binary32
    assert abs(fp64 - got[0]) <= MIXED_TOL * abs(fp64)


@pytest.mark.parametrize("prob", [
    W.atm_problem("fcc", W.Quad(n_u=8, n_v=64, u_rule=2, lam=0.0, r_real=0.0, r_recip=0.0)),
    W.nbody_problem("fcc", 6.0, 5, W.Quad(n_u=32, n_v=48, lam=0.0, r_real=0.0, r_recip=0.0)),
    W.nbody_problem("bcc", 12.0, 2, W.Quad(n_u=8, n_v=32, u_rule=2, lam=0.0, r_real=0.0, r_recip=0.0), scale=1.2),
], ids=["atm-fcc-config3", "fcc-nu6-n5-config4", "bcc-nu12-served"])
def test_mixed_full_size_sampled_lines(ez, oracle_mod, prob):
    _sampled_lines(ez, oracle_mod, prob, 11, 4, MIXED_TOL, prec=ez.EZ_MIXED)


def test_mixed_batch_matches_single(ez):
    probs = [W.nbody_problem("hexagonal", 3.0, 3, W.config2(32)), W.atm_problem("square", W.Quad(
        n_u=4, n_v=8, u_rule=2, lam=1.0, r_real=6, r_recip=6))]
    lats = [ez.Lattice(p.A) for p in probs]
    specs = [ez.sum_spec(p.nu, p.expo) for p in probs]
    quads = [ez.quadrature(p.quad, prec=ez.EZ_MIXED) for p in probs]
    many = ez.ez_lattice_sums(lats, specs, quads)
    for i in range(len(probs)):
        one = ez.ez_lattice_sums([lats[i]], [specs[i]], [quads[i]])
        assert np.array_equal(one[0], many[i])


def test_err_est_bounds_the_quadrature_error(ez):
    # zeta^(2)_{Z^2}(3,3) = Z_6(0) = 4 zeta(3) beta(3), beta(3) = pi^3/32 (Cor. one/two-body)
    exact = 4 * 1.2020569031595942854 * math.pi ** 3 / 32
    L = ez.Lattice(W.lattice("square"))
    errs = []
    for n in (4, 6, 10, 16):
        q = ez.quadrature(W.Quad(n_u=n, n_v=n, u_rule=1, lam=1.0, r_real=6.0, r_recip=6.0))
        v, err = ez.ez_lattice_sum_nbody(L, [3.0, 3.0], q, err_est=True)
        assert v == ez.ez_lattice_sum_nbody(L, [3.0, 3.0], q)  # the estimate does not change the value
        assert abs(v - exact) <= err, (n, v, exact, err)
        errs.append(err)
    # the estimate is the coarse rule's error: it falls geometrically with n (oracle: 1.8, 2.5e-2,
    # 2.7e-6, 1.3e-10 for n = 4, 6, 10, 16)
    assert errs == sorted(errs, reverse=True) and errs[-1] < 1e-9 * exact


@pytest.mark.parametrize("lat", ["square", "hexagonal"])
def test_large_n_sums(ez, oracle_mod, lat):
    """Sec. 4.4, n-body zeta functions zeta^(n)(3,..,3): line-by-line parity with the oracle at
    n = 2, 3, 8, 16; zeta^(2)(3,3) = Z_6(0) (Cor. one/two-body); and for n up to 51 the bound
    0 < zeta^(n) <= Z_3(0)^n, with zeta^(n) / Z_3(0)^n decreasing in n (|Z_3(k)| <= Z_3(0))."""
    for n in (2, 3, 8, 16):
        _compare_with_oracle(ez, oracle_mod, W.nbody_problem(lat, 3.0, n, W.config2(32)))
    A = W.lattice(lat)
    L = ez.Lattice(A)
    q = ez.quadrature(W.config2(64))
    z6 = oracle_mod.epstein_zeta(A, 6.0, np.zeros(2), np.zeros(2), 1.0, 8.0, 8.0).real
    assert ez.ez_lattice_sum_nbody(L, [3.0, 3.0], q) == pytest.approx(z6, rel=1e-13)
    z3 = oracle_mod.epstein_zeta(A, 3.0, np.zeros(2), np.zeros(2), 1.0, 8.0, 8.0).real
    ns = list(range(2, 52))
    vals = ez.ez_lattice_sums([L] * len(ns), [ez.sum_spec([3.0], [[n]]) for n in ns], [q] * len(ns))[:, 0]
    ratio = vals / z3 ** np.array(ns, dtype=float)
    assert np.all(ratio > 0) and np.all(ratio <= 1.0)
    assert np.all(np.diff(ratio) < 0)


# ------------------------------------------------------------------ real (non-integer) exponents
REAL_NU_ZETA = [("Z", [1.5, 2.3, 4.25, -0.7]), ("hexagonal", [0.6, 2.45, 3.3, 5.15]), ("fcc", [-1.3, 2.2, 3.5, 6.5])]


@pytest.mark.parametrize("lat,nus", REAL_NU_ZETA)
def test_epstein_zeta_real_nu(ez, oracle_mod, lat, nus):
    """Def. "Epstein zeta function" at real nu: Gamma(a, t) of non-half-integer orders on the
    device (tables from the backward continued fraction and series) against the oracle."""
    A = W.lattice(lat)
    d = A.shape[0]
    L = ez.Lattice(A)
    rng = np.random.default_rng(23)
    ys = rng.uniform(-0.5, 0.5, (30, d)) @ np.linalg.inv(A)
    lam = abs(np.linalg.det(A)) ** (1.0 / d)
    for nu in nus:
        for x in (np.zeros(d), A @ rng.uniform(-0.5, 0.5, d)):
            re, im = ez.ez_epstein_zeta(L, nu, x, ys)
            for i in range(0, len(ys), 3):
                z = oracle_mod.epstein_zeta(A, nu, x, ys[i], lam, 9.0 * lam, 9.0 / lam)
                assert abs(complex(re[i], im[i]) - z) <= TOL * max(1.0, abs(z)), (lat, nu, i, re[i], z)


REAL_NU_SUMS = [
    W.Problem("Z:real3", W.lattice("Z"), [4.5], [[3]], W.Quad(n_u=12, n_v=1, u_rule=2, lam=1.0, r_real=8, r_recip=8)),
    W.Problem("Z:mixed-orders", W.lattice("Z"), [2.4, 3.7], [[1, 2]], W.Quad(n_u=10, n_v=1, u_rule=2, lam=1.0,
                                                                            r_real=8, r_recip=8)),
    W.Problem("hex:real3", W.lattice("hexagonal"), [3.3], [[3]], W.Quad(n_u=5, n_v=10, u_rule=2, lam=1.0, r_real=6,
                                                                       r_recip=6)),
    W.Problem("sq:below-d", W.lattice("square"), [1.6, 3.1], [[2, 1]], W.Quad(n_u=5, n_v=9, u_rule=2, lam=1.0,
                                                                              r_real=6, r_recip=6)),
    W.Problem("fcc:real2", W.lattice("fcc"), [6.5], [[2]], W.Quad(n_u=3, n_v=6, u_rule=2, lam=1.0, r_real=4.5,
                                                                  r_recip=4.5)),
]


@pytest.mark.parametrize("prob", REAL_NU_SUMS, ids=[p.name for p in REAL_NU_SUMS])
def test_nbody_real_nu_parity(ez, oracle_mod, prob):
    """n-body sums with real exponents (eps-split rule, real Hadamard exponents mu + 2k): every
    quadrature line against the oracle, FP64 form."""
    _compare_with_oracle(ez, oracle_mod, prob)


def test_real_nu_two_body_identity_and_mixed_form(ez, oracle_mod):
    # zeta^(2)(nu1, nu2) = Z_{nu1 + nu2}(0) for real exponents; the mixed form within 1e-10
    A = W.lattice("hexagonal")
    L = ez.Lattice(A)
    q = W.Quad(n_u=14, n_v=24, u_rule=2, lam=0.0, r_real=0.0, r_recip=0.0)
    ref = oracle_mod.epstein_zeta(A, 6.1, np.zeros(2), np.zeros(2), 1.0, 9.0, 9.0).real
    for prec, tol in ((ez.EZ_FP64, 1e-13), (ez.EZ_MIXED, 1e-10)):
        v = ez.ez_lattice_sum_nbody(L, [2.75, 3.35], ez.quadrature(q, prec=prec))
        assert v == pytest.approx(ref, rel=tol)
