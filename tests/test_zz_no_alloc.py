"""The allocation-free Epstein zeta entry point (ez_epstein_zeta_static).

Some callers cannot allocate device memory when they need a value (code inside an
allocator or a memory-pool callback, real-time threads that must stay out of the
driver's allocator, processes whose device memory another framework has reserved).
ez_epstein_zeta_static serves them from a 256 KiB static device array.  This file is
collected last on purpose; it checks, through the C ABI, that two calls in a row give
the values of the allocating entry point ez_epstein_zeta, and that oversized tables are
rejected with a clear error.
"""
import numpy as np
import pytest

from paper_2504_11989_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-13  # the tolerance of the FP64 parity tests


@pytest.fixture(scope="module")
def ez():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2504_11989_gb300 import build, ezeta

    build.build()
    return ezeta


def test_two_calls_in_a_row_match_the_allocating_entry(ez):
    import torch

    rng = np.random.default_rng(2026)
    # a large table first, then a smaller one, so stale contents of the shared static
    # array would show up in the second call
    cases = [("fcc", 6.0, True), ("hexagonal", 3.0, False)]
    for lat_name, nu, x_is_zero in cases:
        A = W.lattice(lat_name)
        d = A.shape[0]
        L = ez.Lattice(A)
        y = rng.uniform(-0.5, 0.5, (300, d)) @ np.linalg.inv(A)
        x = np.zeros(d) if x_is_zero else A @ rng.uniform(-0.5, 0.5, d)
        ref_re, ref_im = ez.ez_epstein_zeta(L, nu, x, y)
        yt = torch.tensor(y, dtype=torch.float64, device="cuda")
        re = torch.full((len(y),), float("nan"), dtype=torch.float64, device="cuda")
        im = torch.full((len(y),), float("nan"), dtype=torch.float64, device="cuda")
        ez.ez_epstein_zeta_static(L, nu, x, yt, re, im)
        got = re.cpu().numpy() + 1j * im.cpu().numpy()
        ref = ref_re + 1j * ref_im
        assert np.all(np.abs(got - ref) <= TOL * np.maximum(np.abs(ref), 1.0)), lat_name


def test_rejects_tables_beyond_the_static_area(ez):
    import torch

    # an elongated unit-density lattice whose tables need ~295 KB (> 256 KiB)
    A = np.diag([0.25, 0.25, 16.0])
    L = ez.Lattice(A)
    y = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    re = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ez.EzError) as e:
        ez.ez_epstein_zeta_static(L, 5.0, np.zeros(3), y, re)
    assert e.value.code == ez.EZ_EINVAL and "static area" in str(e.value)
    # host buffers are refused too (they would need staging memory): by the binding, and by
    # the C ABI itself when called directly
    sq = ez.Lattice(W.lattice("square"))
    with pytest.raises(ValueError):
        ez.ez_epstein_zeta_static(sq, 3.0, np.zeros(2), torch.zeros((2, 2), dtype=torch.float64),
                                  torch.zeros(2, dtype=torch.float64))
    import ctypes

    yh, rh, x0 = np.zeros((2, 2)), np.zeros(2), np.zeros(2)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = ez.lib().ez_epstein_zeta_static(sq.handle, 3.0, x0.ctypes.data_as(dp), ctypes.c_void_p(yh.ctypes.data), 2,
                                         ctypes.c_void_p(rh.ctypes.data), None, None)
    assert rc == ez.EZ_EINVAL
