"""Pins of the dust self-absorption cycles (Sect. 3.2) in the oracle: energy
bookkeeping of every cycle, the fixed point the cycles converge to, and the
limit of dust that is transparent to its own emission."""
import dataclasses

import numpy as np
import pytest

from oracle import emission as E
from oracle import selfabsorb as OSA
from selfabsorb_case import PACKETS_PER_LAMBDA, SEED, stellar_case


@pytest.fixture(scope="module")
def case():
    return stellar_case()


@pytest.fixture(scope="module")
def run(case):
    prob, A, mass, wl = case
    return OSA.self_absorption(prob.grid, A, prob.wl.lam, mass, PACKETS_PER_LAMBDA, SEED, tol=1e-2,
                               max_cycles=12, wl=wl)


def test_pair_reduces_to_the_single_table(case):
    prob, A, mass, _ = case
    lam_em, _ = E.emission_grid()
    one, T1, P1 = E.exact_emission(A, prob.wl.lam, mass)
    two, T2, P2 = E.exact_emission_pair(A, prob.wl.lam, np.zeros((A.shape[0], lam_em.size)), lam_em, mass)
    assert np.array_equal(one, two) and np.array_equal(T1, T2)
    # two tables on disjoint grids act as one table on the joined grid
    rng = np.random.default_rng(2)
    B = rng.random((A.shape[0], lam_em.size)) * A.sum(axis=1, keepdims=True) / lam_em.size
    pair, _, Pp = E.exact_emission_pair(A, prob.wl.lam, B, lam_em, mass)
    joint, _, Pj = E.exact_emission(np.hstack([A, B]), np.concatenate([prob.wl.lam, lam_em]), mass)
    np.testing.assert_allclose(Pp, Pj, rtol=1e-13)
    np.testing.assert_allclose(pair, joint, rtol=1e-11, atol=1e-300)


def test_every_cycle_conserves_energy(case, run):
    prob, A, _, _ = case
    assert run["converged"] and 3 <= run["cycles"] <= 12
    prev = 0.0
    for h in run["history"]:
        # the dust emits what it absorbed of the stars and of itself in the previous cycle
        assert h["emitted"] == pytest.approx(A.sum() + prev, rel=1e-12)
        led = h["ledger"]
        assert led[:, 0].sum() == pytest.approx(h["emitted"], rel=1e-12)
        closure = np.abs(led[:, 0] - led[:, 1] - led[:, 2] - led[:, 3]).sum() / led[:, 0].sum()
        assert closure < 1e-12
        assert h["status"] == 0
        prev = h["absorbed"]
    assert run["absorbed_dust"].sum() == pytest.approx(run["history"][-1]["absorbed"], rel=1e-12)


def test_cycles_reach_the_fixed_point(case, run):
    """If a fraction f of the dust emission is re-absorbed, the absorbed dust
    luminosity D obeys D = f (S + D), so D = f S / (1 - f) at convergence;
    a cycle that dropped or doubled the dust's own heating would not land
    there."""
    prob, A, _, _ = case
    S = A.sum()
    last = run["history"][-1]
    f = last["absorbed"] / last["emitted"]
    assert 0.1 < f < 0.6
    assert last["absorbed"] == pytest.approx(f * S / (1 - f), rel=0.02)
    # the first cycle sees the stellar heating only and re-absorbs less than the fixed point
    assert run["history"][0]["absorbed"] < 0.8 * last["absorbed"]


def test_transparent_dust_converges_at_once(case):
    prob, A, mass, wl = case
    clear = dataclasses.replace(wl, kscale=wl.kscale * 1e-8)
    r = OSA.self_absorption(prob.grid, A, prob.wl.lam, mass, PACKETS_PER_LAMBDA, SEED, tol=1e-2, max_cycles=5,
                            wl=clear)
    h = r["history"]
    assert r["cycles"] == 2 and r["converged"]
    assert h[0]["absorbed"] < 1e-6 * h[0]["emitted"]
    assert h[1]["emitted"] == pytest.approx(h[0]["emitted"], rel=1e-6)


def test_batched_cycles_trace_the_same_packets(case, run):
    """The batch-means option splits every cycle's packets into disjoint
    ranges: the same packets, so the same cycles and tables (to FP64
    summation order); its variance estimate of a cycle's absorbed total
    agrees with the one computed here from the per-packet absorbed records
    of the last cycle (an independent estimate: sum over packets of the
    squared deviations, n/(n-1) corrected, which the batch means approach
    within their own sampling error)."""
    import oracle
    prob, A, mass, wl = case
    b = OSA.self_absorption(prob.grid, A, prob.wl.lam, mass, PACKETS_PER_LAMBDA, SEED, tol=1e-2, max_cycles=12,
                           wl=wl, batches=10)
    assert b["cycles"] == run["cycles"]
    for x, y in zip(b["history"], run["history"]):
        assert x["absorbed"] == pytest.approx(y["absorbed"], rel=1e-12)
        assert x["var_absorbed"] > 0
    np.testing.assert_allclose(b["absorbed_dust"], run["absorbed_dust"], rtol=1e-12, atol=1e-300)
    # the last cycle again, with a record of every packet
    cdf, totals = OSA.cell_cdf(b["emission"])
    npk = np.where(totals > 0, PACKETS_PER_LAMBDA, 0).astype(np.uint64)
    last = _cycle_problem(prob, wl, totals, npk, len(b["history"]) - 1)
    r = oracle.trace(last, peel=False, cell_cdf=cdf, nrec=PACKETS_PER_LAMBDA)
    a = r["records"][..., 2][npk > 0].ravel()
    var_packets = a.size / (a.size - 1.0) * np.sum((a - a.mean()) ** 2)
    assert r["ledger"][:, 1].sum() == pytest.approx(b["history"][-1]["absorbed"], rel=1e-12)
    # ten batches estimate a variance with a relative standard error of about sqrt(2/9) = 0.47
    assert 0.2 < b["history"][-1]["var_absorbed"] / var_packets < 3.0


def _cycle_problem(prob, wl, totals, npk, k):
    from paper_1705_04702_gb300 import workloads as W
    return W.Problem("cycle", prob.grid, W.Source(W.SRC_DUST), dataclasses.replace(wl, lsrc=totals), npk, [],
                     seed=SEED, phase=OSA.PHASE0 + k)
