"""C ABI checks that need no GPU: the library builds for sm_103a, exports every
function declared in include/ezeta.h, and its host-side validation and layout
logic behave as documented (no kernel is launched here)."""
import ctypes
import os
import re
import shutil

import pytest

from paper_2504_11989_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ez():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2504_11989_gb300 import build, ezeta

    build.build()
    return ezeta


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ezeta.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*|long long)\s+(ez_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(ez):
    names = declared_functions()
    assert len(names) >= 10
    L = ez.lib()
    for n in names:
        assert hasattr(L, n), n


def test_lattice_validation(ez):
    with pytest.raises(ez.EzError) as e:
        ez.Lattice([[1.0, 2.0], [0.5, 1.0]])
    assert e.value.code == ez.EZ_EINVAL
    h = ctypes.c_void_p()
    A = (ctypes.c_double * 49)(*([1.0] * 49))
    assert ez.lib().ez_lattice_create(7, A, 1.0, ctypes.byref(h)) == ez.EZ_EINVAL
    assert b"d = 7" in ez.lib().ez_last_error()
    # singular in 4 dimensions (all-ones matrix)
    assert ez.lib().ez_lattice_create(4, A, 1.0, ctypes.byref(h)) == ez.EZ_EINVAL
    lat = ez.Lattice(W.lattice("fcc"))
    assert lat.d == 3


def test_higher_dimensional_lattices(ez):
    """d = 4..6 lattices exist for the Epstein zeta function; the lattice sums (Duffy nodes,
    near part) are built for d <= 3 and refuse them with EZ_EUNSUPPORTED, before any device work."""
    import numpy as np

    for name in ("Z4", "D4", "Z5", "D5", "Z6", "E6"):
        A = W.lattice(name)
        assert abs(abs(np.linalg.det(A)) - 1.0) < 1e-12
        lat = ez.Lattice(A)
        assert lat.d == A.shape[0]
    # the root lattices: Gram matrices with 2 on the diagonal before rescaling
    for name in ("D4", "D5", "E6"):
        A = W.lattice(name, unit_density=False)
        G = A.T @ A
        assert np.allclose(np.diag(G), 2.0) and set(np.round(G[~np.eye(len(G), dtype=bool)], 12)) <= {0.0, -1.0}
    # det of the Cartan matrices: D_n 4, E6 3
    assert abs(np.linalg.det(W.lattice("D4", unit_density=False)) ** 2 - 4.0) < 1e-10
    assert abs(np.linalg.det(W.lattice("E6", unit_density=False)) ** 2 - 3.0) < 1e-10
    spec = ez.sum_spec([5.0], [[2]])
    with pytest.raises(ez.EzError) as e:
        ez.ez_plan_describe(ez.Lattice(W.lattice("D4")), spec, ez.quadrature(W.Quad(n_u=4, n_v=4)))
    assert e.value.code == ez.EZ_EUNSUPPORTED


@pytest.mark.parametrize(
    "d,nu,expo,quad,expect",
    [
        (1, [4.0], [[3]], W.config1(4096), (1, 4096, 1)),
        (2, [3.0], [[3]], W.config2(256), (4, 128, 1)),
        (3, [-1.0, 1.0, 3.0, 5.0], W.ATM_EXPO, W.config3(64, 8), (12, 48, 2)),
        (3, [6.0], [[8]], W.config4(), (12, 32, 1)),
        (2, [4.0], [[2]], W.Quad(n_u=7, n_v=5, u_rule=0), (4, 42, 2)),  # log case picks the eps-split
    ],
)
def test_layout(ez, d, nu, expo, quad, expect):
    assert ez.ez_layout(d, ez.sum_spec(nu, expo), ez.quadrature(quad)) == expect


def test_layout_rejects_hadamard_pole_and_bad_exponents(ez):
    q = ez.quadrature(W.Quad(n_u=8, n_v=1, u_rule=2))
    with pytest.raises(ez.EzError) as e:  # d = 1, nu = (-1, 2): mu_T = 1 - 2 + 1 = 0
        ez.ez_layout(1, ez.sum_spec([-1.0, 2.0], [[1, 1]]), q)
    assert e.value.code == ez.EZ_EDOMAIN
    # a real exponent is planned with the eps-split rule (nu - d is not an odd integer)
    assert ez.ez_layout(2, ez.sum_spec([2.5], [[2]]), ez.quadrature(W.Quad(n_u=8, n_v=4, u_rule=0)))[2] == 2
    with pytest.raises(ez.EzError) as e:
        ez.ez_layout(2, ez.sum_spec([float("nan")], [[2]]), q)
    assert e.value.code == ez.EZ_EINVAL
    with pytest.raises(ez.EzError) as e:
        ez.ez_layout(2, ez.sum_spec([-4.0], [[2]]), q)
    assert e.value.code == ez.EZ_EDOMAIN
    with pytest.raises(ez.EzError) as e:
        ez.ez_layout(2, ez.sum_spec([3.0], [[2]]), ez.quadrature(W.Quad(n_u=8, n_v=300)))
    assert e.value.code == ez.EZ_EINVAL


def test_layout_rejects_bad_part(ez):
    q = ez.quadrature(W.Quad(n_u=8, n_v=8), part=3, n_parts=2)
    with pytest.raises(ez.EzError) as e:
        ez.ez_layout(2, ez.sum_spec([3.0], [[2]]), q)
    assert e.value.code == ez.EZ_EINVAL
    # a valid part plans like the whole sum (same tables and line count)
    whole = ez.ez_layout(2, ez.sum_spec([3.0], [[2]]), ez.quadrature(W.Quad(n_u=8, n_v=8)))
    part = ez.ez_layout(2, ez.sum_spec([3.0], [[2]]), ez.quadrature(W.Quad(n_u=8, n_v=8), part=1, n_parts=2))
    assert part[1:] == whole[1:]


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2504_11989_gb300 import ezeta

    monkeypatch.setattr(ezeta, "_lib", None)
    monkeypatch.setattr(ezeta, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        ezeta.lib()


def test_epstein_zeta_buffer_checks(ez):
    # the C ABI gets bare pointers; the binding rejects every size or device mismatch
    # before a kernel could read or write past the caller's buffers
    import numpy as np
    import torch

    lat = ez.Lattice(W.lattice("square"))
    y = np.zeros((5, 2))
    with pytest.raises(ValueError, match="x has 3"):
        ez.ez_epstein_zeta(lat, 3.0, [0.0, 0.0, 0.0], y)
    with pytest.raises(ValueError, match="shape"):
        ez.ez_epstein_zeta(lat, 3.0, [0.0, 0.0], np.zeros((5, 3)))
    with pytest.raises(ValueError, match="shape"):
        ez.ez_epstein_zeta(lat, 3.0, [0.0, 0.0], np.zeros(7))
    with pytest.raises(ValueError, match="re holds 4"):
        ez.ez_epstein_zeta(lat, 3.0, [0.0, 0.0], y, re=np.zeros(4))
    with pytest.raises(ValueError, match="im holds 2"):
        ez.ez_epstein_zeta(lat, 3.0, [0.0, 0.0], y, re=np.zeros(5), im=np.zeros(2))
    with pytest.raises(ValueError, match="CPU tensors"):
        ez.ez_epstein_zeta(lat, 3.0, [0.0, 0.0], torch.zeros(5, 2, dtype=torch.float64))
    # the allocation-free entry takes CUDA tensors only
    with pytest.raises(ValueError, match="CUDA tensors"):
        ez.ez_epstein_zeta_static(lat, 3.0, [0.0, 0.0], y, np.zeros(5))
    with pytest.raises(ValueError, match="re holds 1"):
        ez.ez_epstein_zeta_static(lat, 3.0, [0.0, 0.0], y, np.zeros(1))


def test_lattice_scale_argument(ez):
    import numpy as np

    A = W.lattice("hexagonal")
    with pytest.raises(ez.EzError) as e:
        ez.Lattice(A, scale=0.0)
    assert e.value.code == ez.EZ_EINVAL
    with pytest.raises(ez.EzError) as e:
        ez.Lattice(A, scale=float("nan"))
    assert e.value.code == ez.EZ_EINVAL
    # the scaled lattice plans like the lattice built from scale * A (the plan sees A only)
    spec = ez.sum_spec([3.0], [[3]])
    q = ez.quadrature(W.Quad(n_u=8, n_v=8))
    a = ez.ez_plan_describe(ez.Lattice(A, scale=1.2), spec, q)
    b = ez.ez_plan_describe(ez.Lattice(1.2 * A), spec, q)
    assert (a.lambda_, a.r_real, a.r_recip, list(a.M)) == (b.lambda_, b.r_real, b.r_recip, list(b.M))
    assert np.allclose(ez.Lattice(A, scale=1.2).A, 1.2 * A)
