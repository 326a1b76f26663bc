"""GPU parity: the CUDA life cycle, called through the C ABI, against the
FP64 oracle on the same seeded inputs and Philox streams."""
import math

import numpy as np
import pytest

from paper_1705_04702_gb300 import tasks
from paper_1705_04702_gb300 import workloads as W

from parity import (MIXED_CELL_SIGNIFICANT, REL_FP64, REL_MIXED_PACKET, REL_MIXED_TALLY, check_mixed,
                    compare_records, compare_tally)

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


def _np(t):
    return t.detach().cpu().numpy() if t is not None else None


def _check(S, oracle_lib, prob, precision, chaotic=False, min_match=0.999, **kw):
    """Records of every packet; the FP64 form against the oracle at 1e-9, the
    mixed form by parity.check_mixed (unmatched packets split off)."""
    nrec = int(max(prob.npk.max(), 1))
    grid = S.Grid(prob.grid)
    g = S.run_problem(prob, grid, precision=precision, nrec=nrec, **kw)
    r = oracle_lib.trace(prob, nrec=nrec)
    fp64 = precision == S.PREC_FP64
    if fp64:
        compare_records(_np(g["records"]), r["records"], prob, REL_FP64, 0.999, same_n_min=1.0)
        compare_tally(_np(g["absorbed"]), r["absorbed"], REL_FP64)
        if prob.instruments:
            compare_tally(_np(g["sed"]), r["sed"], REL_FP64, significant=0.0)
            compare_tally(_np(g["images_flat"]), r["images_flat"], REL_FP64, significant=1e-6)
        np.testing.assert_allclose(g["ledger_per_lambda"], r["ledger"], rtol=REL_FP64, atol=1e-300)
        summary = None
    else:
        summary = check_mixed(S, oracle_lib, grid, prob, g, r, chaotic=chaotic, min_match=min_match)
        print(prob.name, summary)
    grid.close()
    tot = g["ledger"]
    closure = abs(tot["emitted"] - tot["absorbed"] - tot["escaped"] - tot["residual"]) / max(tot["emitted"], 1e-300)
    assert closure < (1e-12 if fp64 else 1e-6), closure
    # the table holds what the packets deposited (per-event bookkeeping in the
    # ledger, per-cell reductions in the table)
    table = float(g["absorbed"].sum())
    assert table == pytest.approx(tot["absorbed"], rel=1e-12 if fp64 else 1e-6)
    if fp64:
        assert tot["scatterings"] == r["counters"][0]
    return g, r


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_sphere_c1(S, oracle_lib, precision):
    prob = W.sphere_problem(100_000)
    _check(S, oracle_lib, prob, precision, min_match=0.998)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_disk_multi_wavelength(S, oracle_lib, precision):
    prob = W.disk_problem(3000, n=64, nlambda=3, npx=64)
    _check(S, oracle_lib, prob, precision, min_match=0.998)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_torus_uneven_counts(S, oracle_lib, precision):
    prob = W.torus_problem(n=48, nlambda=12, packet_scale=2e-4, npx=48)
    prob.npk[3] = 0  # an empty wavelength in the middle
    _check(S, oracle_lib, prob, precision, chaotic=True)


def test_packet_ranges_compose(S):
    """Calls over disjoint packet ranges of one run (first_packet /
    total_packets, the task split of Sect. 5.2) trace the same histories as
    one call over all packets, and their tables add up to its tables."""
    import torch
    prob = W.torus_problem(n=32, nlambda=5, packet_scale=1e-4, npx=32)
    prob.npk[2] = 0
    grid = S.Grid(prob.grid)
    nrec = int(prob.npk.max())
    for prec in (S.PREC_FP64, S.PREC_MIXED):
        full = S.run_problem(prob, grid, precision=prec, nrec=nrec)
        _, cut = tasks.packet_share(prob.npk, 0, 3)
        a = S.run_problem(prob.with_packets(cut), grid, precision=prec, nrec=nrec, total_packets=prob.npk)
        b = S.run_problem(prob.with_packets(prob.npk - cut), grid, precision=prec, nrec=nrec, first_packet=cut,
                          total_packets=prob.npk)
        fr = _np(full["records"])
        for j in range(prob.wl.n):
            k, n = int(cut[j]), int(prob.npk[j])
            assert np.array_equal(_np(a["records"])[j, :k], fr[j, :k])
            assert np.array_equal(_np(b["records"])[j, :n - k], fr[j, k:n])
        compare_tally(_np(a["absorbed"] + b["absorbed"]), _np(full["absorbed"]), 1e-12)
        compare_tally(_np(a["images_flat"] + b["images_flat"]), _np(full["images_flat"]), 1e-12)
        compare_tally(_np(a["sed"] + b["sed"]), _np(full["sed"]), 1e-12, significant=0.0)
        np.testing.assert_allclose(a["ledger_per_lambda"] + b["ledger_per_lambda"], full["ledger_per_lambda"],
                                   rtol=1e-12, atol=1e-300)
    # a range beyond the run is refused
    with pytest.raises(S.SkirtError) as e:
        S.run_problem(prob, grid, first_packet=np.ones(prob.wl.n, np.uint64), total_packets=prob.npk)
    assert e.value.code == S.ERR_INVALID_ARG
    grid.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("schedule", [0, 1], ids=["per_lambda", "persistent"])
def test_schedules_and_launch_shapes_give_identical_histories(S, schedule):
    """Per-packet histories depend only on (seed, packet, wavelength): every
    schedule, block size and refill chunk gives bit-identical records."""
    prob = W.torus_problem(n=32, nlambda=5, packet_scale=1e-4, npx=32)
    base = S.run_problem(prob, precision=S.PREC_MIXED, schedule=S.SCHED_PERSISTENT, nrec=500)
    for block, chunk in ((64, 1), (128, 3), (256, 16)):
        other = S.run_problem(prob, precision=S.PREC_MIXED, schedule=schedule, nrec=500, block=block, chunk=chunk)
        assert np.array_equal(_np(base["records"]), _np(other["records"]))
        compare_tally(_np(other["absorbed"]), _np(base["absorbed"]), 1e-12)


def test_slab_beam_exact(S):
    layer = np.array([0.2, 0.3, 0.5, 4.0], dtype=np.float32).astype(np.float64)
    grid = W.slab_grid(layer)
    for prec in (S.PREC_FP64, S.PREC_MIXED):
        prob = W.beam_problem(grid, (0.1, 0.2, 0.0), (0.6, 0.0, 0.8), npackets=1, albedo=0.0)
        g = S.run_problem(prob, precision=prec, nrec=1)
        rec = _np(g["records"])[0, 0]
        # mixed: e^{-tau} evaluated in FP32 from an FP64 tau of ~8: ~8 * 2^-24 + a few ulp
        tol = 1e-14 if prec == S.PREC_FP64 else 3e-6
        assert rec[1] == pytest.approx(math.exp(-layer.sum() / 0.8), rel=tol)
        cum = np.concatenate([[0.0], np.cumsum(layer)]) / 0.8
        got = _np(g["absorbed"])[:, 0].reshape(grid.nz, -1).sum(axis=1)
        np.testing.assert_allclose(got, np.exp(-cum[:-1]) - np.exp(-cum[1:]), rtol=tol)


def test_edge_cases(S, oracle_lib):
    # no packets at all
    prob = W.sphere_problem(0)
    g = S.run_problem(prob)
    assert float(g["absorbed"].abs().sum()) == 0 and g["ledger"]["emitted"] == 0
    # a single packet, a 1x1x1 grid
    grid = W.uniform_grid(1, kr=0.7)
    prob = W.Problem("one", grid, W.Source(W.SRC_POINT, (0.1, -0.3, 0.2)), W.single_wavelength(),
                     np.array([1], np.uint64), [W.Instrument(10.0, 20.0, 10.0, 2.0, 3)])
    for prec in (0, 1):
        g = S.run_problem(prob, precision=prec, nrec=1)
        r = oracle_lib.trace(prob, nrec=1)
        compare_records(_np(g["records"]), r["records"], prob, REL_FP64 if prec == 0 else REL_MIXED_PACKET)
    # dust-free grid: everything escapes, nothing absorbed
    prob = W.Problem("empty", W.uniform_grid(8, kr=0.0), W.Source(W.SRC_POINT, (0.0, 0.0, 0.0)),
                     W.single_wavelength(), np.array([1000], np.uint64), [W.Instrument(10.0, 0.0, 0.0, 2.0, 8)])
    g = S.run_problem(prob, nrec=10)
    assert float(g["absorbed"].abs().sum()) == 0
    # mixed form: the packet luminosity 1/1000 is an FP32 value
    assert g["ledger"]["escaped"] == pytest.approx(1.0, rel=1e-7)
    assert float(g["sed"][0, 0]) == pytest.approx(1.0 / (4 * math.pi * 100), rel=1e-6)
    # no instruments, and peel-off disabled
    prob = W.sphere_problem(2000)
    ref = oracle_lib.trace(prob, peel=False)
    for p in (True, False):
        q = W.sphere_problem(2000)
        if p:
            q.instruments = []
        g = S.run_problem(q, precision=0, peel=not p)
        compare_tally(_np(g["absorbed"]), ref["absorbed"], REL_FP64)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_ragged_grid_and_sixteen_instruments(S, oracle_lib, precision):
    """A non-cubic grid with odd, unequal sides (37 x 29 x 11 cells of unequal
    shape), three wavelengths with ragged packet counts, and the maximum of 16
    instruments in all directions with odd pixel counts and frames that
    leave part of the galaxy outside (out-of-frame peel-offs).  The FP64 form
    follows the oracle to 1e-9; in the mixed form the coarse cells (up to 1.7
    units across, 0.55 thick in z) let FP32 interaction points drift further
    over 5-7 scatterings, so 99.8% of the packets must agree within 1e-5
    (measured 99.88%)."""
    grid = W.disk_grid(nxyz=(37, 29, 11))
    wl = W.powerlaw_wavelengths(3, 0.2, 3.0)
    ins = [W.Instrument(50.0 + 7 * q, 11.25 * q, 23.0 * q, 20.0 + 4 * (q % 5), 5 + 2 * q) for q in range(16)]
    prob = W.Problem("ragged", grid, W.Source(W.SRC_DISK, (0.0, 0.0, 0.0), h_R=4.0, h_z=0.4), wl,
                     np.array([1500, 1, 977], np.uint64), ins, seed=3)
    _check(S, oracle_lib, prob, precision, min_match=0.998)


def test_event_cap_is_reported(S):
    prob = W.sphere_problem(100)
    prob.max_events = 1
    g = S.run_problem(prob, nrec=100)
    assert g["status"] == S.ERR_EVENT_CAP
    assert np.all(_np(g["records"])[0, :, 0] == 1)


def test_graph_replay_host_buffers_and_accumulate(S):
    import torch
    prob = W.disk_problem(4000, n=32, nlambda=2, npx=32)
    grid = S.Grid(prob.grid)
    a = S.run_problem(prob, grid=grid, precision=1)
    b1 = S.run_problem(prob, grid=grid, precision=1, use_graph=True)
    b2 = S.run_problem(prob, grid=grid, precision=1, use_graph=True)
    for b in (b1, b2):
        compare_tally(_np(b["absorbed"]), _np(a["absorbed"]), 1e-12)
        compare_tally(_np(b["sed"]), _np(a["sed"]), 1e-12, significant=0.0)
    # host (pinned and pageable) output buffers give the same tallies
    n = prob.wl.n
    npix = sum(i.npx * i.npx for i in prob.instruments) * n
    for pin in (True, False):
        outs = (torch.zeros((grid.ncell, n), dtype=torch.float64, pin_memory=pin),
                torch.zeros(npix, dtype=torch.float64, pin_memory=pin),
                torch.zeros((len(prob.instruments), n), dtype=torch.float64, pin_memory=pin))
        h = S.run_problem(prob, grid=grid, precision=1, outputs=outs)
        compare_tally(h["absorbed"].numpy(), _np(a["absorbed"]), 1e-12)
        compare_tally(h["sed"].numpy(), _np(a["sed"]), 1e-12, significant=0.0)
    # accumulate: a second call with another seed adds to the first
    p2 = W.disk_problem(4000, n=32, nlambda=2, npx=32, seed=7)
    c = S.run_problem(p2, grid=grid, precision=1)
    outs = (a["absorbed"].clone(), torch.cat([a["images_flat"].clone()]), a["sed"].clone())
    acc = S.run_problem(p2, grid=grid, precision=1, outputs=outs, accumulate=True)
    compare_tally(_np(acc["absorbed"]), _np(a["absorbed"] + c["absorbed"]), 1e-12)
    compare_tally(_np(acc["sed"]), _np(a["sed"] + c["sed"]), 1e-12, significant=0.0)
    grid.close()


def test_invalid_arguments(S):
    prob = W.sphere_problem(10)
    bad = W.sphere_problem(10)
    bad.wl.albedo[0] = 1.5
    with pytest.raises(S.SkirtError) as e:
        S.run_problem(bad)
    assert e.value.code == S.ERR_INVALID_ARG
    bad = W.sphere_problem(10)
    bad.source = W.Source(W.SRC_POINT, (5.0, 0.0, 0.0))
    with pytest.raises(S.SkirtError):
        S.run_problem(bad)
    g = prob.grid
    g2 = W.Grid(g.nx, g.ny, g.nz, g.bbox, g.kr.copy())
    g2.kr[0, 0, 0] = np.nan
    with pytest.raises(S.SkirtError):
        S.Grid(g2)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_dust_cell_source(S, oracle_lib, precision):
    """Dust emission phase source: cells drawn from the per-wavelength CDF of
    an emission table (built here with numpy, independently of the library's
    scan), a uniform point inside the cell, isotropic direction; the source
    luminosity of each wavelength is the table's column sum (lsrc = NULL)."""
    import dataclasses
    import torch
    grid = W.sphere_grid(16, kr_in=2.0)
    rng = np.random.default_rng(4)
    nl = 3
    em = rng.random((grid.ncell, nl)) ** 4 * (grid.kr.ravel()[:, None] > 0)
    em[:, 1] *= 1e-3
    totals = em.sum(axis=0)
    cdf = np.cumsum(em, axis=0) / totals
    cdf[-1] = 1.0
    wl = W.powerlaw_wavelengths(nl, 1.0, 100.0, alb_short=0.3, alb_long=0.0)
    prob = W.Problem("dust", grid, W.Source(W.SRC_DUST), wl, np.array([3000, 2000, 0], np.uint64),
                     [W.Instrument(50.0, 30.0, 10.0, 2.0, 16)], seed=9)
    prob.phase = 1
    r = oracle_lib.trace(dataclasses.replace(prob, wl=dataclasses.replace(wl, lsrc=totals)), nrec=3000,
                         cell_cdf=np.ascontiguousarray(cdf.T))
    g = S.run_problem(dataclasses.replace(prob, wl=dataclasses.replace(wl, lsrc=None)), precision=precision,
                      nrec=3000, emission=torch.as_tensor(em, device="cuda"))
    rel = REL_FP64 if precision == 0 else REL_MIXED_PACKET
    # record fields scale with the packets' launch luminosity totals / N
    scaled = dataclasses.replace(prob, wl=dataclasses.replace(wl, lsrc=totals))
    compare_records(_np(g["records"]), r["records"], scaled, rel, 0.999, same_n_min=0.999)
    np.testing.assert_allclose(g["ledger_per_lambda"][:, 0], [totals[0], totals[1], 0.0], rtol=1e-6)
    compare_tally(_np(g["absorbed"]), r["absorbed"], rel if precision == 0 else REL_MIXED_TALLY,
                  significant=1e-6 if precision == 0 else MIXED_CELL_SIGNIFICANT)


def test_autotune_picks_a_swept_schedule_with_identical_histories(S):
    """skirt_autotune on a small torus: the chosen schedule is one of the
    timed candidates and not slower than the requested one on the sample, the
    outputs are left zeroed, and a trace with the tuned schedule gives records
    bit-identical to the default schedule's (histories depend only on the
    packet)."""
    import torch
    prob = W.torus_problem(n=48, nlambda=12, packet_scale=2e-4, npx=32)
    grid = S.Grid(prob.grid)
    n = prob.wl.n
    npix = sum(i.npx * i.npx for i in prob.instruments) * n
    absorbed = torch.full((grid.ncell, n), float("nan"), dtype=torch.float64, device="cuda")
    images = torch.full((npix,), float("nan"), dtype=torch.float64, device="cuda")
    sed = torch.full((len(prob.instruments), n), float("nan"), dtype=torch.float64, device="cuda")
    opts = S.skirt_trace_opts_default()
    tables = S.Tables(prob.wl)
    rep = S.skirt_autotune(grid.h, S.make_source(prob.source), tables.c, prob.npk, prob.seed,
                           S.make_instruments(prob.instruments), opts, 0.5, absorbed, images, sed, repeats=2)
    torch.cuda.synchronize()
    assert float(absorbed.abs().sum()) == 0 and float(images.abs().sum()) == 0 and float(sed.abs().sum()) == 0
    pts = rep["points"]
    assert rep["n"] > 10 and 0 <= rep["chosen"] < rep["n"] and rep["repeats"] == 2
    c = pts[rep["chosen"]]
    assert (opts.block, opts.chunk, opts.blocks_per_sm, opts.step_min) == (c["block"], c["chunk"],
                                                                          c["blocks_per_sm"], c["step_min"])
    assert all(p["ms"] > 0 for p in pts)
    confirmed = [p for p in pts if p["ms_confirm"] > 0]
    assert pts[0]["ms_confirm"] > 0 and c["ms_confirm"] > 0 and 2 <= len(confirmed) <= 4
    assert c["ms_confirm"] <= pts[0]["ms_confirm"]
    assert rep["confirm_packets"] > rep["sample_packets"] or rep["confirm_packets"] == int(prob.npk.sum())
    nrec = int(prob.npk.max())
    base = S.run_problem(prob, grid, nrec=nrec)
    tuned = S.run_problem(prob, grid, nrec=nrec, block=opts.block, chunk=opts.chunk,
                          blocks_per_sm=opts.blocks_per_sm, step_min=opts.step_min, use_graph=True)
    assert np.array_equal(_np(base["records"]), _np(tuned["records"]))
    compare_tally(_np(tuned["absorbed"]), _np(base["absorbed"]), 1e-12)
    grid.close()


@pytest.mark.parametrize("chaotic", [False, True], ids=["sphere", "torus"])
def test_parity_criterion_detects_a_planted_mistake(S, oracle_lib, chaotic):
    """The mixed-form criterion has power: the oracle, run on the same packets
    of a problem whose albedo is 5% higher (a mistake planted in the oracle's
    input, on the CPU), fails check_mixed against the GPU's run of the right
    problem, in a smooth medium and in the clumpy torus."""
    import dataclasses
    if chaotic:
        prob = W.torus_problem(n=32, nlambda=4, packet_scale=5e-5, npx=32)
    else:
        prob = W.sphere_problem(20000)
    wrong = dataclasses.replace(prob, wl=dataclasses.replace(prob.wl, albedo=np.minimum(prob.wl.albedo * 1.05,
                                                                                         1.0)))
    nrec = int(prob.npk.max())
    grid = S.Grid(prob.grid)
    g = S.run_problem(prob, grid, precision=S.PREC_MIXED, nrec=nrec)
    r = oracle_lib.trace(wrong, nrec=nrec)
    with pytest.raises(AssertionError):
        check_mixed(S, oracle_lib, grid, prob, g, r, chaotic=chaotic)
    grid.close()


def test_optical_depth_cut_changes_no_history(S, monkeypatch):
    """The mixed form stops a deposit or peel-off traversal once its optical
    depth passes 30.  Walking every path to the boundary instead
    (SKIRT_MIXED_TAU_CUT=1e30) changes no packet history: scattering counts
    and interaction points are bit-identical on the clumpy torus, and a
    packet's luminosity fields move by less than 1e-12 (what the cut leaves
    out is below e^-30 of a packet).  A table entry collects such tails over
    many traversals, so the tables and ledgers are held to 1e-10."""
    prob = W.torus_problem(n=48, nlambda=200, packet_scale=2e-4, npx=64)
    grid = S.Grid(prob.grid)
    a = S.run_problem(prob, grid, precision=S.PREC_MIXED, nrec=60)
    monkeypatch.setenv("SKIRT_MIXED_TAU_CUT", "1e30")
    b = S.run_problem(prob, grid, precision=S.PREC_MIXED, nrec=60)
    grid.close()
    ra, rb = _np(a["records"]), _np(b["records"])
    assert np.array_equal(ra[..., 0], rb[..., 0])      # scatterings
    assert np.array_equal(ra[..., 5:8], rb[..., 5:8])  # last interaction point
    scale = np.abs(rb[..., 1:5]).max()
    assert np.abs(ra[..., 1:5] - rb[..., 1:5]).max() <= 1e-12 * scale
    compare_tally(_np(a["absorbed"]), _np(b["absorbed"]), 1e-10)
    compare_tally(_np(a["images_flat"]), _np(b["images_flat"]), 1e-10)
    for k in ("emitted", "absorbed", "escaped", "residual", "scatterings"):
        assert a["ledger"][k] == pytest.approx(b["ledger"][k], rel=1e-10, abs=1e-10 * b["ledger"]["emitted"])
