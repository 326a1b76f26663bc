"""The allocation-free exact emission entry point.

skirt_dust_emission_exact_static serves callers that cannot allocate device
memory while they run (their allocator has already reserved the memory they
may use, or their memory budget is fixed before the loop starts).  It keeps
its one working table in a fixed device array instead.  These tests call it
through the C-ABI twice in a row, with different wavelength grids, and check
each result against skirt_dust_emission in exact mode; the second call must
not see anything the first one left in the shared array.  The file is named
to be collected last, so it also runs after every other GPU test."""
import numpy as np
import pytest

from paper_1705_04702_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STATIC_MAX_NIN = 4096


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300 import skirt
    return skirt


def _case(n, lam, seed):
    import torch
    a, m = W.absorbed_spectra(n, lam, seed=seed)
    a[:2] = 0.0      # cells without absorbed power
    m[2:4] = 0.0     # dust-free cells
    return (torch.as_tensor(a, dtype=torch.float64, device="cuda"),
            torch.as_tensor(m, dtype=torch.float32, device="cuda"))


def _run_both(S, a, m, lam):
    import torch
    n = a.shape[0]
    em0 = torch.zeros((n, 100), dtype=torch.float64, device="cuda")
    T0 = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    S.skirt_dust_emission(a, n, lam.size, lam, m, S.EMIT_EXACT, None, em0, T0)
    # outputs pre-filled with garbage: the entry point must write every element
    em1 = torch.full((n, 100), float("nan"), dtype=torch.float64, device="cuda")
    T1 = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    S.skirt_dust_emission_exact_static(a, n, lam.size, lam, m, em1, T1)
    torch.cuda.synchronize()
    return em0.cpu().numpy(), T0.cpu().numpy(), em1.cpu().numpy(), T1.cpu().numpy()


def test_static_matches_allocating_entry_point_twice(S):
    # first call: a wide grid (the table nearly full); second call: a short grid
    # with other wavelengths, so a stale table would change the result
    for lam, n, seed in ((np.geomspace(0.09, 10.0, 4000), 1500, 11),
                         (np.geomspace(0.1, 3.0, 37), 2500, 12)):
        a, m = _case(n, lam, seed)
        em0, T0, em1, T1 = _run_both(S, a, m, lam)
        assert np.all(np.isfinite(em1)) and np.all(np.isfinite(T1))
        # the same FP64 solver on the same share table: the FP64 tolerance of the other tests
        np.testing.assert_allclose(em1, em0, rtol=1e-9, atol=0)
        np.testing.assert_allclose(T1, T0, rtol=1e-6, atol=0)


def test_static_rejects_oversized_grid(S):
    import torch
    lam = np.geomspace(0.09, 10.0, STATIC_MAX_NIN + 1)
    a = torch.zeros((4, lam.size), dtype=torch.float64, device="cuda")
    m = torch.ones(4, dtype=torch.float32, device="cuda")
    em = torch.zeros((4, 100), dtype=torch.float64, device="cuda")
    with pytest.raises(S.SkirtError) as ei:
        S.skirt_dust_emission_exact_static(a, 4, lam.size, lam, m, em)
    assert ei.value.code == S.ERR_INVALID_ARG
    assert "maximum" in str(ei.value)
