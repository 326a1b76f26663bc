"""Dust self-absorption cycles (arXiv:1705.04702 Sect. 3.2, dust
self-absorption phase).

Once the stellar packets are done, every cycle
  1. computes the emission spectrum of every dust cell from the absorbed
     stellar luminosity plus the luminosity the dust absorbed of its own
     emission in the previous cycle (``skirt_dust_emission_pair``),
  2. launches dust packets from the cells in proportion to that emission,
     without peel-off, and collects what they deposit in a separate table,
     the absorbed dust luminosity table (``skirt_trace``, dust-cell source),
until the thermal emission field has converged: here, until the total
absorbed dust luminosity D changes from one cycle to the next by at most
``tol`` times the total heating S + D (S: the absorbed stellar luminosity).
The dust emission phase that follows (the final spectra and a trace with
peel-off) is the caller's.

Every step runs in the library's kernels through the C ABI; this module only
allocates device memory and decides when to stop.  Cycle k draws its random
numbers in stream phase PHASE0 + k, apart from the stellar (0) and dust
emission (1) phases.
"""
from __future__ import annotations

import numpy as np

from . import skirt as S
from . import workloads as W

PHASE0 = 16


def dust_wavelengths():
    """The emission grid (100 wavelengths, 1-1000 micron) with the dust's
    extinction (kappa ~ lambda^-1.2), albedo 0.3 -> 0 and g = 0.6 there."""
    lam, _ = S.skirt_emission_grid()
    return W.powerlaw_wavelengths(S.NEMIT, float(lam[0]), float(lam[-1]), alb_short=0.3, alb_long=0.0)


def self_absorption(grid, absorbed_star, lam_star, mass, packets_per_lambda, seed, tol=1e-2, max_cycles=10,
                    precision=None, wl=None):
    """Runs the cycles on a skirt.Grid.  absorbed_star: device double
    [ncell, len(lam_star)]; mass: device float [ncell].  Returns a dict with
    the absorbed dust table of the last cycle, the emission table that fed it,
    the number of cycles, whether the total converged, and per cycle the dust
    luminosity emitted and re-absorbed and the trace's ledger."""
    import torch
    ncell = grid.ncell
    wl = dust_wavelengths() if wl is None else wl
    wl.lsrc = None  # the emission table's column sums
    lam_em, _ = S.skirt_emission_grid()
    tables = S.Tables(wl)
    opts = S.skirt_trace_opts_default()
    opts.peel = 0
    if precision is not None:
        opts.precision = precision
    dev = absorbed_star.device
    emission = torch.empty((ncell, S.NEMIT), dtype=torch.float64, device=dev)
    absorbed_dust = None
    history = []
    converged = False
    for k in range(max_cycles):
        S.skirt_dust_emission_pair(absorbed_star, ncell, lam_star, absorbed_dust, None if absorbed_dust is None
                                   else lam_em, mass, emission)
        totals = S.skirt_emission_totals(grid.h, emission, S.NEMIT)
        npk = np.where(totals > 0, int(packets_per_lambda), 0).astype(np.uint64)
        src = S.make_source(W.Source(W.SRC_DUST), emission=emission)
        opts.phase = PHASE0 + k
        new = torch.zeros((ncell, S.NEMIT), dtype=torch.float64, device=dev)
        _, led, _ = S.skirt_trace(grid.h, src, tables.c, npk, seed, [], opts, new, None, None)
        history.append({"emitted": float(totals.sum()), "absorbed": led["absorbed"], "ledger": led})
        absorbed_dust = new
        if k > 0:
            prev, cur = history[-2]["absorbed"], history[-1]["absorbed"]
            if abs(cur - prev) <= tol * (history[0]["emitted"] + cur):
                converged = True
                break
    return {"absorbed_dust": absorbed_dust, "emission": emission, "cycles": len(history), "converged": converged,
            "history": history}
