"""Sec. 5 on the GPU: the lattice sums of the fcc/bcc stability scan (Z_n(0), Z_m(0) and the
ATM energy of the unit-nearest-neighbour lattices) against the oracle, and the phase boundary
they give: fcc stable without three-body forces, bcc beyond a critical ATM coupling, the
boundary moving to larger coupling with pressure -- strongly for the (12,6) Lennard-Jones
potential, hardly for (8,4)."""
import numpy as np
import pytest

from paper_2504_11989_gb300 import phase as P
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


def test_coefficients_match_the_oracle(ez, oracle_mod):
    q = W.Quad(n_u=3, n_v=8, u_rule=2, lam=1.0, r_real=5.0, r_recip=5.0)
    for name in P.UNIT_NN:
        c = P.coefficients(ez, name, 12, 6, ez.quadrature(q))
        A = W.lattice(name, unit_density=False)
        for nu, got in ((12, c.z_n), (6, c.z_m)):
            ref = oracle_mod.epstein_zeta(A, float(nu), np.zeros(3), np.zeros(3), 1.0, 8.0, 8.0).real
            assert got == pytest.approx(ref, rel=1e-13)
        ref = oracle_mod.atm_energy(oracle_mod.nbody(W.Problem(name, A, list(W.ATM_NU), W.ATM_EXPO, q), threads=16))
        assert c.e_atm == pytest.approx(ref, rel=1e-13)


def test_phase_boundary(ez):
    q = ez.quadrature(W.Quad(n_u=4, n_v=24, u_rule=2, lam=0.0, r_real=0.0, r_recip=0.0))
    pressures = (0.0, 1.0, 5.0)
    lam_c = {}
    for n, m in ((12, 6), (8, 4)):
        f, b = (P.coefficients(ez, name, n, m, q) for name in P.UNIT_NN)
        for p in pressures:
            assert P.enthalpy_gap(f, b, 0.0, p) > 0.0  # fcc without three-body forces
        lam_c[n, m] = [P.critical_coupling(f, b, p) for p in pressures]
        assert all(x is not None and x > 0.0 for x in lam_c[n, m])
        assert np.all(np.diff(lam_c[n, m]) > 0.0)  # pressure favours fcc
    assert lam_c[12, 6][-1] - lam_c[12, 6][0] > 0.1
    assert lam_c[8, 4][-1] - lam_c[8, 4][0] < 0.02
