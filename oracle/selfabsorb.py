"""Dust self-absorption cycles, FP64 oracle -- TEST INFRASTRUCTURE ONLY
(see oracle/__init__.py).

Method (arXiv:1705.04702, Sect. 3.2, dust self-absorption phase): after the
stellar emission phase, the emission spectrum of every dust cell is computed
from the absorbed stellar luminosity; dust packets are launched from the cells
according to these emission luminosities, with no peel-off, and their
absorption goes into a second table, the absorbed dust luminosity table; the
cycle repeats, each time with the emission computed from both tables, until
the thermal emission field has converged.  Reading used here: convergence
when the total absorbed dust luminosity D changes between two cycles by at
most ``tol`` times the total heating S + D (S: the absorbed stellar
luminosity, which the first cycle emits), so that dust transparent to its own
emission stops at once; every cycle starts a fresh dust table; cycle k uses
random-stream phase PHASE0 + k; the dust-cell source takes the emission
table's column sums as its luminosities and gives packets only to
wavelengths with emission.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_1705_04702_gb300 import workloads as W

from . import trace
from .emission import emission_grid, exact_emission, exact_emission_pair

PHASE0 = 16


def dust_wavelengths():
    lam, _ = emission_grid()
    return W.powerlaw_wavelengths(lam.size, float(lam[0]), float(lam[-1]), alb_short=0.3, alb_long=0.0)


def cell_cdf(emission):
    """Per-wavelength cumulative distribution over the cells [nlambda][ncell]
    of an emission table [ncell][nlambda] (zero rows for dark wavelengths)."""
    totals = emission.sum(axis=0)
    cdf = np.zeros((emission.shape[1], emission.shape[0]))
    for j in np.nonzero(totals > 0)[0]:
        cdf[j] = np.cumsum(emission[:, j]) / totals[j]
        cdf[j, -1] = 1.0
    return cdf, totals


def self_absorption(grid, absorbed_star, lam_star, mass, packets_per_lambda, seed, tol=1e-2, max_cycles=10,
                    wl=None, batches=1):
    """The cycles on a workloads.Grid; returns the absorbed dust table of the
    last cycle, the emission that fed it, the cycle count, whether the total
    converged, and per cycle the emitted and re-absorbed dust luminosity.

    batches > 1 traces every cycle's packets as that many disjoint packet
    ranges (the same packets; the table is their sum) and adds the Monte
    Carlo error estimates of the batch means method: per cycle the variance
    of the absorbed total ("var_absorbed"), and the variance of every entry of
    the last cycle's table ("var_absorbed_dust")."""
    lam_em, _ = emission_grid()
    wl = dust_wavelengths() if wl is None else wl
    absorbed_dust = None
    history = []
    converged = False
    emission = None
    for k in range(max_cycles):
        if absorbed_dust is None:
            emission, _, _ = exact_emission(absorbed_star, lam_star, mass)
        else:
            emission, _, _ = exact_emission_pair(absorbed_star, lam_star, absorbed_dust, lam_em, mass)
        cdf, totals = cell_cdf(emission)
        npk = np.where(totals > 0, int(packets_per_lambda), 0).astype(np.uint64)
        prob = W.Problem("dust self-absorption cycle", grid, W.Source(W.SRC_DUST),
                         dataclasses.replace(wl, lsrc=totals), npk, [], seed=seed, phase=PHASE0 + k)
        if batches <= 1:
            r = trace(prob, peel=False, cell_cdf=cdf)
            var_tab = None
        else:
            r, var_tab = _batched_trace(prob, cdf, int(packets_per_lambda), batches)
        history.append({"emitted": float(totals.sum()), "absorbed": float(r["ledger"][:, 1].sum()),
                        "ledger": r["ledger"], "status": r["status"]})
        if var_tab is not None:
            history[-1]["var_absorbed"] = float(r["var_total"])
        absorbed_dust = r["absorbed"]
        if k > 0:
            prev, cur = history[-2]["absorbed"], history[-1]["absorbed"]
            if abs(cur - prev) <= tol * (history[0]["emitted"] + cur):
                converged = True
                break
    out = {"absorbed_dust": absorbed_dust, "emission": emission, "cycles": len(history), "converged": converged,
           "history": history}
    if batches > 1:
        out["var_absorbed_dust"] = var_tab
    return out


def _batched_trace(prob, cdf, npk, batches):
    """The trace of prob as `batches` disjoint packet ranges: the summed
    result, plus the batch-means variance estimate of every table entry and
    of the absorbed total (variance of the sum = B/(B-1) sum_b (x_b - x/B)^2)."""
    edges = np.linspace(0, npk, batches + 1).round().astype(np.int64)
    parts = [trace(prob, int(a), int(b), peel=False, cell_cdf=cdf) for a, b in zip(edges[:-1], edges[1:])]
    tab = np.sum([p["absorbed"] for p in parts], axis=0)
    led = np.sum([p["ledger"] for p in parts], axis=0)
    B = float(batches)
    var_tab = B / (B - 1.0) * np.sum([(p["absorbed"] - tab / B) ** 2 for p in parts], axis=0)
    tot = np.array([p["ledger"][:, 1].sum() for p in parts])
    var_tot = B / (B - 1.0) * np.sum((tot - tot.sum() / B) ** 2)
    status = 0
    for p in parts:
        status |= p["status"]
    return {"absorbed": tab, "ledger": led, "status": status, "var_total": var_tot}, var_tab
