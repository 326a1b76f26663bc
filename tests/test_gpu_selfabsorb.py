"""GPU parity of the dust self-absorption cycles (Sect. 3.2): the exact
emission from two absorbed tables, the emission totals, and the whole cycle
loop, against the FP64 oracle on the same inputs and Philox streams."""
import math

import numpy as np
import pytest

from oracle import emission as E
from oracle import selfabsorb as OSA
from paper_1705_04702_gb300 import workloads as W
from parity import K_SIGMA, REL_MIXED_TALLY, compare_tally
from selfabsorb_case import PACKETS_PER_LAMBDA, SEED, stellar_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1705_04702_gb300 import build
    build.build()
    from paper_1705_04702_gb300 import skirt
    return skirt


@pytest.fixture(scope="module")
def case():
    return stellar_case()


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_pair_emission_matches_oracle(S):
    import torch
    lam_a = np.geomspace(0.09, 10.0, 60)
    lam_b, _ = S.skirt_emission_grid()
    a, m = W.absorbed_spectra(2000, lam_a, seed=7)
    rng = np.random.default_rng(8)
    b = rng.random((2000, lam_b.size)) * a.sum(axis=1, keepdims=True) / lam_b.size
    em = torch.zeros((2000, 100), dtype=torch.float64, device="cuda")
    S.skirt_dust_emission_pair(_dev(a, torch.float64), 2000, lam_a, _dev(b, torch.float64), lam_b,
                               _dev(m, torch.float32), em)
    ref, _, _ = E.exact_emission_pair(a, lam_a, b, lam_b, m.astype(np.float64))
    g = em.cpu().numpy()
    big = ref > 1e-9 * ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(g[big], ref[big], rtol=1e-9)
    np.testing.assert_allclose(g.sum(axis=1), a.sum(axis=1) + b.sum(axis=1), rtol=1e-12)
    # without the second table: the single-table solve, bit for bit
    one = torch.zeros_like(em)
    S.skirt_dust_emission_pair(_dev(a, torch.float64), 2000, lam_a, None, None, _dev(m, torch.float32), one)
    single = torch.zeros_like(em)
    S.skirt_dust_emission(_dev(a, torch.float64), 2000, lam_a.size, lam_a, _dev(m, torch.float32), S.EMIT_EXACT,
                          None, single)
    assert torch.equal(one, single)


def test_emission_totals(S, case):
    import torch
    prob, A, mass, _ = case
    grid = S.Grid(prob.grid)
    rng = np.random.default_rng(3)
    em = rng.random((grid.ncell, 100)) ** 3
    em[:, :5] = 0.0  # dark wavelengths
    t = S.skirt_emission_totals(grid.h, _dev(em, torch.float64), 100)
    np.testing.assert_allclose(t, em.sum(axis=0), rtol=1e-13)
    assert np.all(t[:5] == 0)
    grid.close()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_cycles_match_oracle(S, case, precision):
    """The whole loop against the oracle's loop.  The FP64 form follows it to
    rounding.  In the mixed form a dust packet whose history diverges (the
    clumpy torus amplifies FP32 rounding), or whose cell is drawn from a CDF
    shifted by an earlier cycle's differences, is a different Monte Carlo
    sample: the differences are bounded by K_SIGMA standard deviations of the
    difference of two independent runs, with the oracle's batch-means error
    estimates (10 packet ranges per cycle), summed over the cycles that feed
    a result; the last cycle's table also moves with its total emission."""
    import torch
    from paper_1705_04702_gb300.selfabsorb import self_absorption
    prob, A, mass, wl = case
    ref = OSA.self_absorption(prob.grid, A, prob.wl.lam, mass, PACKETS_PER_LAMBDA, SEED, tol=1e-2, max_cycles=12,
                              wl=wl, batches=10)
    grid = S.Grid(prob.grid)
    out = self_absorption(grid, _dev(A, torch.float64), prob.wl.lam, _dev(mass, torch.float32), PACKETS_PER_LAMBDA,
                          SEED, tol=1e-2, max_cycles=12, precision=precision, wl=wl)
    grid.close()
    assert out["converged"] and out["cycles"] == ref["cycles"]
    fp64 = precision == 0
    var_sum = 0.0
    for g, r in zip(out["history"], ref["history"]):
        if fp64:
            assert g["emitted"] == pytest.approx(r["emitted"], rel=1e-9)
            assert g["absorbed"] == pytest.approx(r["absorbed"], rel=1e-6)
        else:
            # cycle k emits S + D_{k-1}: its difference is the previous cycles' absorbed differences
            assert abs(g["emitted"] - r["emitted"]) <= K_SIGMA * np.sqrt(2 * var_sum) + 1e-9 * r["emitted"]
            var_sum += r["var_absorbed"]
            assert abs(g["absorbed"] - r["absorbed"]) <= K_SIGMA * np.sqrt(2 * var_sum) + REL_MIXED_TALLY * r["absorbed"]
        led = g["ledger"]
        closure = abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["residual"]) / led["emitted"]
        assert closure < (1e-12 if fp64 else 1e-6)
    # the last cycle's absorbed dust table, cell by cell
    gt = out["absorbed_dust"].cpu().numpy()
    rt = ref["absorbed_dust"]
    if fp64:
        compare_tally(gt, rt, 1e-6, significant=1e-6, l1=1e-6)
        return
    shift = abs(out["history"][-1]["emitted"] - ref["history"][-1]["emitted"]) / ref["history"][-1]["emitted"]
    # the mixed form ends a deposit traversal once its optical depth passes 30
    # and drops deposits below the FP32 range: at most e^-30 of the cycle's
    # emitted luminosity goes missing from any cell
    cut = math.exp(-30.0) * ref["history"][-1]["emitted"]
    bound = K_SIGMA * np.sqrt(2 * ref["var_absorbed_dust"]) + (2 * shift + REL_MIXED_TALLY) * np.abs(rt) + cut
    bad = np.abs(gt - rt) > bound + 1e-300
    assert not bad.any(), (int(bad.sum()), np.abs(gt - rt)[bad][:5], bound[bad][:5])
