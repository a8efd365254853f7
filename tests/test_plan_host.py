"""Host-side planning checked without a GPU (ez_plan_describe): the partition of a sum into
parts, the 3-D block decomposition and its shared-memory bound, the default splitting
parameter, and the mixed form's precision thresholds, the last two against incomplete gamma
values from mpmath (independent of the library's own Gamma code)."""
import math
import shutil
import os

import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W

AUTO = dict(lam=0.0, r_real=0.0, r_recip=0.0)


@pytest.fixture(scope="module")
def ez():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_11989_gb300 import build, ezeta

    build.build()
    return ezeta


def _plan(ez, prob, prec=0, **kw):
    L = ez.Lattice(prob.A)
    return ez.ez_plan_describe(L, ez.sum_spec(prob.nu, prob.expo), ez.quadrature(prob.quad, prec=prec, **kw))


def _phi(a, t):
    """Phi_a(t) = t^{-a} Gamma(a, t), any real a (mpmath, 30 digits)."""
    import mpmath

    mpmath.mp.dps = 30
    return float(mpmath.gammainc(a, t) * mpmath.power(t, -a))


PROBS = [
    W.nbody_problem("Z", 4.0, 3, W.Quad(n_u=300, n_v=1, **AUTO)),
    W.nbody_problem("hexagonal", 3.0, 3, W.Quad(n_u=20, n_v=17, **AUTO)),
    W.atm_problem("square", W.Quad(n_u=6, n_v=10, u_rule=2, **AUTO)),
    W.nbody_problem("fcc", 6.0, 3, W.Quad(n_u=32, n_v=48, **AUTO)),
    W.atm_problem("sc", W.Quad(n_u=8, n_v=64, u_rule=2, **AUTO)),
    W.atm_problem("bcc", W.Quad(n_u=3, n_v=7, u_rule=2, **AUTO)),
    W.nbody_problem("sc", 9.0, 2, W.Quad(n_u=4, n_v=64, u_rule=2, **AUTO)),
]


@pytest.mark.parametrize("prob", PROBS, ids=lambda p: p.name)
@pytest.mark.parametrize("n_parts", [2, 3, 7])
def test_parts_tile_the_far_lines(ez, prob, n_parts):
    """The parts' line ranges are disjoint, contiguous and cover every far line (d <= 2)
    or line group (d = 3: the four sectors of one axis and u node)."""
    whole = _plan(ez, prob)
    d = prob.A.shape[0]
    units = (3 if d == 3 else whole.n_sectors) * whole.n_u_total
    assert (whole.line_lo, whole.line_hi) == (0, units)
    hi = 0
    for k in range(n_parts):
        p = _plan(ez, prob, part=k, n_parts=n_parts)
        assert p.line_lo == hi and p.line_hi >= p.line_lo
        hi = p.line_hi
        if d >= 2:
            assert p.n_far_items == (p.line_hi - p.line_lo) * p.n_chunks
    assert hi == units


@pytest.mark.parametrize("prec", [0, 1])
def test_3d_blocks_fit_two_per_sm(ez, prec):
    """d = 3: the v2 rows of a block are covered by the chunks, and a block's dynamic shared
    memory stays within 98 KB (two blocks per SM) unless the smallest chunk (8 rows) is
    already larger."""
    reqs = W.serving_mix(120, W.SEED_BASE + 5, 1.0)
    seen = 0
    for r in reqs:
        if r.d != 3:
            continue
        p = W.request_problem(r)
        info = _plan(ez, p, prec=prec)
        n_v = p.quad.n_v
        assert info.n_chunks * info.vchunk >= n_v > (info.n_chunks - 1) * info.vchunk
        assert info.far_smem_bytes <= 98 * 1024 or info.vchunk == min(n_v, 8)
        assert max(info.M) <= 16
        seen += 1
    assert seen > 10


@pytest.mark.parametrize("lat,d", [("Z", 1), ("square", 2), ("hexagonal", 2), ("sc", 3), ("fcc", 3), ("bcc", 3)])
@pytest.mark.parametrize("prec", [0, 1])
def test_default_splitting_parameter(ez, lat, d, prec):
    """lam = 0: 2 V (d = 1), 3 V^{1/2} (d = 2), 4.5 V^{1/3} (FP64) or 4 V^{1/3} (mixed) in 3-D,
    lowered only as far as the real-space box half-width 16 requires; the cutoffs are
    sqrt(T/pi) lam^{+-1} with T = 45 (FP64) or 36 (mixed)."""
    A = W.lattice(lat, scale=1.17)
    V = abs(np.linalg.det(A))
    prob = W.nbody_problem(lat, 4.0 if d < 3 else 6.0, 3, W.Quad(n_u=8, n_v=8, **AUTO), scale=1.17)
    info = _plan(ez, prob, prec=prec)
    f = {1: 2.0, 2: 3.0, 3: 4.0 if prec else 4.5}[d]
    T = 36.0 if prec else 45.0
    want = f * V ** (1.0 / d)
    assert info.lambda_ <= want * (1 + 1e-12)
    rows = np.linalg.norm(np.linalg.inv(A), axis=1)
    R = math.sqrt(T / math.pi) * info.lambda_
    assert info.r_real == pytest.approx(R, rel=1e-12)
    assert info.r_recip == pytest.approx(math.sqrt(T / math.pi) / info.lambda_, rel=1e-12)
    M = [math.ceil(R * rn + 1e-9) for rn in rows]
    assert list(info.M)[:d] == M and max(M) <= 16
    if info.lambda_ < want * (1 - 1e-12):  # lowered: the box would exceed 16 at the default
        assert max(math.ceil(math.sqrt(T / math.pi) * want * rn + 1e-9) for rn in rows) > 16


@pytest.mark.parametrize("prob", [PROBS[1], PROBS[3], PROBS[4], PROBS[6]], ids=lambda p: p.name)
def test_mixed_thresholds_against_mpmath(ez, prob):
    """Mixed form: beyond t_mix every reciprocal order has |Phi_a(t)| t <= 1e-7 and beyond t_mid
    |Phi_a(t)| <= 1e-6 (on the 0.25 grid the planner scans); one grid step earlier the bound
    fails for some order (the thresholds are the first grid points that hold)."""
    info = _plan(ez, prob, prec=1)
    d = prob.A.shape[0]
    orders = [0.5 * (d - nu) for nu in prob.nu]
    tm, td = float(info.t_mix), float(info.t_mid)
    for t in np.arange(tm, tm + 8.0, 0.25):
        assert all(abs(_phi(a, t)) * t <= 1e-7 for a in orders), t
    assert any(abs(_phi(a, tm - 0.25)) * (tm - 0.25) > 1e-7 for a in orders)
    for t in np.arange(td, tm, 0.25):
        assert all(abs(_phi(a, t)) <= 1e-6 for a in orders), t
    if td < tm:
        assert any(abs(_phi(a, td - 0.25)) > 1e-6 for a in orders)


@pytest.mark.parametrize("prob", [PROBS[3], PROBS[4], PROBS[5]], ids=lambda p: p.name)
def test_mixed_binary32_shells_against_mpmath(ez, prob):
    """Mixed form: m_hp[i] is the first |m_i| at which every real-space order's term is below
    1e-8 of its value at the shortest lattice vector (|z| >= |m_i| / |row_i(A^{-1})|)."""
    info = _plan(ez, prob, prec=1)
    A = prob.A
    lam = info.lambda_
    shifts = [np.array(m) - 2 for m in np.ndindex(5, 5, 5)]
    dmin2 = min(float(np.sum((A @ m) ** 2)) for m in shifts if np.any(m))
    Ai = np.linalg.inv(A)
    orders = [0.5 * nu for nu in prob.nu]
    ref = [abs(_phi(a, math.pi * dmin2 / lam ** 2)) for a in orders]

    def small(m, rn2):
        return all(abs(_phi(a, math.pi * (m * m / rn2) / lam ** 2)) <= 1e-8 * r for a, r in zip(orders, ref))

    for i in range(3):
        rn2 = float(np.sum(Ai[i] ** 2))
        m = info.m_hp[i]
        if m <= info.M[i]:
            assert small(m, rn2)
        if m > 1:
            assert not small(m - 1, rn2)


def test_plan_describe_errors_and_fp64_thresholds(ez):
    """Bad arguments fail as the sums would (part out of range, real-space box wider than
    16); the FP64 form has no binary32 thresholds, the mixed form's lie inside the table."""
    prob = W.nbody_problem("fcc", 6.0, 3, W.Quad(n_u=4, n_v=8, **AUTO))
    with pytest.raises(RuntimeError):
        _plan(ez, prob, part=3, n_parts=3)
    with pytest.raises(RuntimeError):
        _plan(ez, W.nbody_problem("fcc", 6.0, 3, W.Quad(n_u=4, n_v=8, lam=1.0, r_real=40.0, r_recip=4.5)))
    info = _plan(ez, prob, prec=0)
    assert info.t_mix > 1e38 and info.t_mid > 1e38
    mixed = _plan(ez, prob, prec=1)
    assert 0.5 < mixed.t_mid <= mixed.t_mix < 40.0
    assert all(1 <= mixed.m_hp[i] <= mixed.M[i] + 1 for i in range(3))


def _axis_reflection_invariant(A, radius=3):
    """Whether every reflection x_i -> -x_i maps the point set A Z^d onto itself, decided on
    the points A n with |n_j| <= radius (a point set test, independent of any basis algebra)."""
    d = A.shape[0]
    grids = np.meshgrid(*[np.arange(-radius, radius + 1)] * d, indexing="ij")
    n = np.stack([g.ravel() for g in grids])
    P = A @ n
    Ainv = np.linalg.inv(A)
    for i in range(d):
        R = P.copy()
        R[i] *= -1.0
        c = Ainv @ R
        if np.max(np.abs(c - np.rint(c))) > 1e-9:
            return False
    return True


def _near_counts(d, ell):
    """Multi-indices alpha in N^d with |alpha| = 2k, k <= ell: all of them, and the all-even ones."""
    full = sum(math.comb(2 * k + d - 1, d - 1) for k in range(ell + 1))
    even = sum(math.comb(k + d - 1, d - 1) for k in range(ell + 1))
    return full, even


def _rot3(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q * np.sign(np.diag(r))


NEAR_LATTICES = [
    ("Z", W.lattice("Z")),
    ("square", W.lattice("square")),
    ("hexagonal", W.lattice("hexagonal")),
    ("oblique", np.array([[1.0, 0.37], [0.0, 1.1]])),
    ("sc", W.lattice("sc")),
    ("fcc", W.lattice("fcc")),
    ("bcc", W.lattice("bcc")),
    ("orthorhombic", np.diag([1.0, 1.3, 0.8])),
    ("triclinic", np.array([[1.0, 0.3, 0.2], [0.0, 1.0, 0.1], [0.0, 0.0, 1.0]])),
    ("rotated sc", _rot3(5)),
]


@pytest.mark.parametrize("ell", [1, 4])
@pytest.mark.parametrize("name,A", NEAR_LATTICES, ids=[n for n, _ in NEAR_LATTICES])
def test_near_multi_indices_follow_axis_reflections(ez, name, A, ell):
    """The near part's Taylor expansion of the regular part of Z (Sec. 3, meromorphic
    continuation; order 2 ell, Sec. 4.1) keeps
    every alpha with even |alpha| <= 2 ell; on a lattice that each axis reflection maps onto
    itself the regular part is even in every component, its odd-alpha coefficients vanish
    and only the all-even alpha are kept.  The count must follow the point set's symmetry,
    not the basis: a rotated simple cubic lattice keeps them all."""
    d = A.shape[0]
    spec = ez.sum_spec(list(W.ATM_NU), [list(r) for r in W.ATM_EXPO])
    q = ez.quadrature(W.Quad(n_u=4, n_v=8, u_rule=2, ell=ell, **AUTO))
    info = ez.ez_plan_describe(ez.Lattice(A), spec, q)
    full, even = _near_counts(d, ell)
    want = even if _axis_reflection_invariant(A) else full
    assert info.n_alpha == want
    assert _axis_reflection_invariant(A) == (name not in ("oblique", "triclinic", "rotated sc"))
    far = ez.ez_plan_describe(ez.Lattice(A), spec, ez.quadrature(W.Quad(n_u=4, n_v=8, u_rule=1, **AUTO)))
    assert far.n_alpha == 0
