"""The adaptive u integration (Sec. 3: standard adaptive quadrature with recursive interval
subdivision) on the GPU, against the oracle: the same sums on a converged fixed rule with the
same v rule, cutoffs and near part, so that only the u integration differs; and, for the
paper's plain adaptive route for nu_i >= d (no eps-split), the two-body identity
zeta^(2)(nu1, nu2) = Z_{nu1+nu2}(0)."""
import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ez():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_11989_gb300 import build, ezeta

    build.build()
    return ezeta


CASES = [  # (problem with the adaptive rule's settings, converged fixed-rule reference)
    (W.nbody_problem("hexagonal", 3.0, 3, W.Quad(n_u=8, n_v=24, u_rule=1, lam=1.0, r_real=6, r_recip=6)), 48),
    (W.atm_problem("square", W.Quad(n_u=8, n_v=20, u_rule=2, lam=1.0, r_real=6, r_recip=6)), 24),
    (W.Problem("fcc:real", W.lattice("fcc"), [5.5], [[3]], W.Quad(n_u=6, n_v=10, u_rule=2, lam=1.0, r_real=4.5,
                                                                  r_recip=4.5)), 20),
]


@pytest.mark.parametrize("prob,n_ref", CASES, ids=[c[0].name for c in CASES])
def test_adaptive_matches_converged_fixed_rule(ez, oracle_mod, prob, n_ref):
    q = prob.quad
    ref_prob = W.Problem(prob.name, prob.A, prob.nu, prob.expo,
                         W.Quad(n_u=n_ref, n_v=q.n_v, u_rule=q.u_rule, eps=q.eps, ell=q.ell, lam=q.lam,
                                r_real=q.r_real, r_recip=q.r_recip))
    ref = oracle_mod.nbody(ref_prob, threads=16)
    L = ez.Lattice(prob.A)
    spec = ez.sum_spec(prob.nu, prob.expo)
    used = []
    for tol in (1e-8, 1e-12):
        v, err, n_u = ez.ez_lattice_sum_adaptive(L, spec, ez.quadrature(q), tol, 40)
        scale = np.abs(ref[: len(v)])
        assert np.all(np.abs(v - ref[: len(v)]) <= 2 * tol * scale + 1e-14 * scale), (prob.name, tol, v, ref)
        assert np.all(err <= 10 * tol * scale) and np.all(np.isfinite(err))
        used.append(n_u)
    assert used[1] >= used[0]  # a tighter tolerance never refines less (analytic cases close at once)


def test_plain_adaptive_route_for_nu_above_d(ez, oracle_mod):
    # nu_i >= d with nu_i - d not odd: the paper integrates u on [0, 1/2] adaptively (u_rule 1,
    # no eps-split); the u^{nu - d} behaviour at u = 0 is resolved by bisection
    A = W.lattice("square")
    L = ez.Lattice(A)
    nus = [2.5, 3.2]
    q = ez.quadrature(W.Quad(n_u=8, n_v=32, u_rule=1, lam=0.0, r_real=0.0, r_recip=0.0))
    v, err, n_u = ez.ez_lattice_sum_adaptive(L, ez.sum_spec(nus, [[1, 1]]), q, 1e-10, 60)
    z = oracle_mod.epstein_zeta(A, sum(nus), np.zeros(2), np.zeros(2), 1.0, 9.0, 9.0).real
    assert v[0] == pytest.approx(z, rel=2e-9)
    assert n_u > 16


def test_adaptive_argument_checks(ez):
    L = ez.Lattice(W.lattice("square"))
    spec = ez.sum_spec([3.0], [[2]])
    q = ez.quadrature(W.config2(16))
    for tol, rounds in ((0.0, 10), (1.5, 10), (1e-8, 1), (1e-8, 61)):
        with pytest.raises(ez.EzError) as e:
            ez.ez_lattice_sum_adaptive(L, spec, q, tol, rounds)
        assert e.value.code == ez.EZ_EINVAL
    with pytest.raises(ez.EzError) as e:
        ez.ez_lattice_sum_adaptive(L, spec, ez.quadrature(W.config2(16), part=0, n_parts=2), 1e-8, 10)
    assert e.value.code == ez.EZ_EINVAL
