"""Parity at full size: the 256^3 exponential-disk workload with 1e8 packets,
traced in the launch configuration the benchmark times (mixed form,
persistent launch replayed from a CUDA graph).  The oracle replays the first
packets of the same streams one by one; the tallies are checked through
properties that hold at any size."""
import math

import numpy as np
import pytest

from paper_1705_04702_gb300 import workloads as W

from parity import (REL_MIXED_PACKET, REL_MIXED_TALLY, compare_records, compare_tally, compare_tally_mc, rebin,
                    rebin_factor, record_sigma_check, scattering_counts_agree, unmatched)

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


def test_disk_1e8_packets_sampled(S, oracle_lib):
    prob = W.disk_problem(100_000_000, n=256, nlambda=1, npx=512)
    nrec = 3000
    g = S.run_problem(prob, precision=S.PREC_MIXED, schedule=S.SCHED_PERSISTENT, nrec=nrec, use_graph=True)
    r = oracle_lib.trace(prob, 0, nrec, nrec=nrec)
    compare_records(g["records"].cpu().numpy(), r["records"], prob, REL_MIXED_PACKET, 0.999, same_n_min=0.999)

    led = g["ledger"]
    assert g["status"] == S.OK and led["status_bits"] == 0
    # every packet was launched with L0 = 1/N
    assert led["emitted"] == pytest.approx(1.0, rel=1e-6)
    closure = abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["residual"]) / led["emitted"]
    assert closure < 1e-6
    # the absorbed table holds the deposits the ledger books
    assert float(g["absorbed"].sum()) == pytest.approx(led["absorbed"], rel=1e-6)
    assert float(g["absorbed"].min()) >= 0.0
    # the SED of every instrument is its image plus the out-of-frame peel-offs
    for q, img in enumerate(g["images"]):
        s_img = float(img.sum())
        assert s_img <= float(g["sed"][q, 0]) * (1 + 1e-12)
        assert s_img >= 0.9 * float(g["sed"][q, 0])
    # work counters match the oracle's per-packet averages on the sample
    c = r["counters"] / nrec
    assert led["scatterings"] / 1e8 == pytest.approx(c[0], rel=0.05)
    assert led["peel_steps"] / 1e8 == pytest.approx(c[3], rel=0.05)
    # the face-on SED is dominated by direct starlight: flux ~ L e^{-tau}/(4 pi d^2)
    F = 1.0 / (4 * math.pi * 100.0 ** 2)
    assert 0.3 * F < float(g["sed"][0, 0]) < 1.5 * F


def test_disk_1e7_packets_full_grid(S):
    """The bench's workload and launch configuration (mixed form, persistent
    launch from a CUDA graph) at 1e7 packets against the oracle run over the
    same packets on every host core.  The first 1e5 packets: >= 99.9% match
    (same scatterings, every record field within 1e-5).  Tables: every
    absorbed cell and every rebinned pixel block holding >= 1e-4 of its
    table's total within 1e-4 plus the Monte Carlo allowance of the <= 0.1%
    unmatched packets (parity.compare_tally_mc, with the batch-means variance
    over the oracle workers' packet ranges); SEDs and ledger within 1e-4."""
    from oracle_pool import trace_all_cores
    n = 10_000_000
    nrec = 100_000
    spec = {"maker": "disk_problem", "kwargs": {"npackets": n, "n": 256, "nlambda": 1, "npx": 512}}
    ref = trace_all_cores(spec, n, nrec=nrec)
    prob = W.disk_problem(n, n=256, nlambda=1, npx=512)
    g = S.run_problem(prob, precision=S.PREC_MIXED, schedule=S.SCHED_PERSISTENT, use_graph=True, nrec=nrec)
    assert g["status"] == S.OK and ref["status"] == 0
    report = {"oracle_cores": ref["cores"]}
    fails = []

    def check(name, fn):
        try:
            report[name] = fn()
        except AssertionError as e:
            fails.append((name, str(e)[:300]))

    small = prob.with_packets(nrec)
    check("records", lambda: compare_records(g["records"].cpu().numpy(), ref["records"], small, REL_MIXED_PACKET,
                                             0.999, same_n_min=0.999))
    check("absorbed", lambda: compare_tally_mc(g["absorbed"].cpu().numpy(), ref["absorbed"], ref["absorbed_var"],
                                               REL_MIXED_TALLY, 1e-4))
    off = 0
    B = float(ref["cores"])
    for q, ins in enumerate(prob.instruments):
        k = ins.npx * ins.npx
        b = rebin_factor(prob, ins)
        gi = rebin(g["images"][q].cpu().numpy(), b)
        ri = rebin(ref["images"][off:off + k].reshape(ins.npx, ins.npx, 1), b)
        parts = [rebin(p[off:off + k].reshape(ins.npx, ins.npx, 1), b) for p in ref["images_parts"]]
        var = B / (B - 1.0) * sum((p - ri / B) ** 2 for p in parts)
        off += k
        report[f"image{q}_bin"] = b
        check(f"image{q}", lambda gi=gi, ri=ri, var=var: compare_tally_mc(gi, ri, var, REL_MIXED_TALLY, 1e-4))
    check("sed", lambda: compare_tally(g["sed"].cpu().numpy(), ref["sed"], REL_MIXED_TALLY, significant=0.0))
    check("ledger", lambda: np.testing.assert_allclose(g["ledger_per_lambda"], ref["ledger"], rtol=REL_MIXED_TALLY))
    print(report, fails)
    assert not fails, fails


def _check_full(S, oracle_lib, prob, nrec, min_match=0.999, same_n_min=0.999, chaotic=False):
    g = S.run_problem(prob, precision=S.PREC_MIXED, schedule=S.SCHED_PERSISTENT, nrec=nrec, use_graph=True)
    r = oracle_lib.trace(prob, 0, nrec, nrec=nrec)
    gr = g["records"].cpu().numpy()
    sample = prob.with_packets(np.minimum(prob.npk, nrec))
    if chaotic:
        # diverged histories are other Monte Carlo samples of the same process:
        # the scattering counts follow the oracle's distribution, and the
        # unmatched packets' shares of the ledger and SEDs differ by at most
        # K_SIGMA standard deviations
        p = scattering_counts_agree(gr, r["records"], sample)
        um = unmatched(gr, r["records"], sample, REL_MIXED_PACKET)
        record_sigma_check(gr, r["records"], sample, um)
        print("chi2 p", p, "unmatched", um.mean())
    else:
        compare_records(gr, r["records"], prob, REL_MIXED_PACKET, min_match, same_n_min=same_n_min)
    led = g["ledger"]
    assert g["status"] == S.OK and led["status_bits"] == 0
    # every wavelength launched its full luminosity (lsrc = 1 per wavelength)
    np.testing.assert_allclose(g["ledger_per_lambda"][:, 0], np.where(prob.npk > 0, prob.wl.lsrc, 0.0), rtol=1e-6)
    closure = abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["residual"]) / led["emitted"]
    assert closure < 1e-6
    assert float(g["absorbed"].sum()) == pytest.approx(led["absorbed"], rel=1e-6)
    # per-wavelength work counters: scatterings per packet of the sample
    c = r["counters"] / int(np.minimum(prob.npk, nrec).sum())
    assert led["scatterings"] / prob.total_packets == pytest.approx(c[0], rel=0.1)
    return g


def test_disk_40_wavelengths_1e7_per_wavelength_sampled(S, oracle_lib):
    """The precision form at scale: 40 wavelengths x 1e7 packets (4e8 packets)."""
    prob = W.disk_problem(10_000_000, n=256, nlambda=40, npx=512)
    _check_full(S, oracle_lib, prob, 300, 0.999)


def test_torus_batched_full_sampled(S, oracle_lib):
    """The batched form at scale: the clumpy torus, 200 wavelengths with
    uneven counts (7.5e8 packets) in one persistent graph launch.  The
    single-cell clumps (100x density) amplify FP32 rounding differences from
    event to event, more so the finer the grid, while the FP64 form follows
    the oracle exactly (next test).  The sampled packets (the first 60 of
    every wavelength) are checked statistically: scattering-count
    distribution, and the unmatched packets' ledger and SED shares within
    K_SIGMA."""
    prob = W.torus_problem(n=256, nlambda=200, npx=512)
    assert prob.total_packets > 5e8
    _check_full(S, oracle_lib, prob, 60, chaotic=True)


def test_torus_256_fp64_histories_follow_the_oracle(S, oracle_lib):
    """The same torus, the first 60 packets of every wavelength in the FP64
    form (histories do not depend on how many other packets run): every
    history has the oracle's scatterings; FP64 rounding-order differences,
    amplified by the clumps over ~20 events, leave 99% of the records within
    1e-9 (measured 99.57%) and 99.9% within 1e-7."""
    from parity import REL_FP64
    prob = W.torus_problem(n=256, nlambda=200, npx=64)
    nrec = 60
    small = prob.with_packets(np.minimum(prob.npk, nrec))
    g = S.run_problem(small, precision=S.PREC_FP64, nrec=nrec)
    r = oracle_lib.trace(small, 0, nrec, nrec=nrec)
    rec = g["records"].cpu().numpy()
    compare_records(rec, r["records"], small, REL_FP64, 0.99, same_n_min=1.0)
    compare_records(rec, r["records"], small, 1e-7, 0.999, same_n_min=1.0)


@pytest.fixture(scope="module")
def disk_tree():
    return W.disk_octree()


def test_disk_octree_8m_leaves_sampled(S, oracle_lib, disk_tree):
    """The ERIS-sized octree: the exponential dust disk refined by dust mass
    into 8.25M leaves (levels 4 to 11, at most 13 levels), 1e7 packets in the
    mixed form in one graph launch; the oracle replays the first 1000 packets
    (its own tree and finest-lattice path listing).  Then the first 300
    packets in the FP64 form follow the oracle to 1e-9."""
    from parity import REL_FP64
    tree = disk_tree
    assert 8.0e6 < tree.ncell < 8.5e6 and tree.max_level == 13
    prob = W.octree_problem(tree, 10_000_000, npx=512)
    grid = S.Grid(tree)
    g = _check_full_on(S, oracle_lib, prob, grid, 1000, 0.998)
    assert float(g["absorbed"].min()) >= 0.0
    small = prob.with_packets(300)
    g = S.run_problem(small, grid, precision=S.PREC_FP64, nrec=300)
    r = oracle_lib.trace(small, 0, 300, nrec=300)
    compare_records(g["records"].cpu().numpy(), r["records"], small, REL_FP64, 1.0, same_n_min=1.0)
    grid.close()


def test_disk_octree_40_wavelengths_sampled(S, oracle_lib, disk_tree):
    """The same tree at 40 wavelengths (0.1-5 micron), 1e6 packets each: the
    wavelength-major accumulation over 8.25M leaves and its transpose into the
    [leaf, wavelength] table (2.6 GB); the oracle replays the first 40
    packets of every wavelength."""
    prob = W.octree_problem(disk_tree, 1_000_000, nlambda=40, npx=128)
    grid = S.Grid(disk_tree)
    g = _check_full_on(S, oracle_lib, prob, grid, 40, 0.995)
    np.testing.assert_allclose(g["ledger_per_lambda"][:, 0], prob.wl.lsrc, rtol=1e-6)
    np.testing.assert_allclose(g["absorbed"].sum(dim=0).cpu().numpy(), g["ledger_per_lambda"][:, 1], rtol=1e-6)
    grid.close()


def _check_full_on(S, oracle_lib, prob, grid, nrec, min_match):
    g = S.run_problem(prob, grid, precision=S.PREC_MIXED, schedule=S.SCHED_PERSISTENT, nrec=nrec, use_graph=True)
    r = oracle_lib.trace(prob, 0, nrec, nrec=nrec)
    compare_records(g["records"].cpu().numpy(), r["records"], prob, REL_MIXED_PACKET, min_match, same_n_min=0.999)
    led = g["ledger"]
    assert g["status"] == S.OK and led["status_bits"] == 0
    closure = abs(led["emitted"] - led["absorbed"] - led["escaped"] - led["residual"]) / led["emitted"]
    assert closure < 1e-6
    assert float(g["absorbed"].sum()) == pytest.approx(led["absorbed"], rel=1e-6)
    c = r["counters"] / int(np.minimum(prob.npk, nrec).sum())
    assert led["scatterings"] / prob.total_packets == pytest.approx(c[0], rel=0.1)
    return g


def test_learned_form_full_grid_sampled(S, oracle_lib):
    """The learned form as configured: the full 256^3 clumpy torus (16.8M
    cells, 200 wavelengths; the absorbed table of the whole 7.5e8-packet
    stellar trace): band features and the exact emission on every cell, the
    oracle on 2000 sampled heated cells; energy exact on every cell; the
    surrogate (trained on 1e6 cells with the default 200 epochs of batch
    2048) energy-exact on every cell; after the guard's fallback the median
    error below 0.5%, the 99th percentile below 1%, at most 10 of the 6.7M
    heated cells above 2% and none above 3% (measured: 0 to 2 cells above
    2%, the largest 1.7-2.4% depending on the training sample: a few
    isolated cells, which neither more epochs nor a tighter guard remove)."""
    import torch
    from oracle import emission as E
    prob = W.torus_problem(n=256, nlambda=200, npx=64)
    grid = S.Grid(prob.grid)
    ncell, nl = grid.ncell, prob.wl.n
    absorbed = torch.zeros((ncell, nl), dtype=torch.float64, device="cuda")
    opts = S.skirt_trace_opts_default()
    opts.peel = 0
    tables = S.Tables(prob.wl)
    S.skirt_trace(grid.h, S.make_source(prob.source), tables.c, prob.npk, prob.seed, [], opts, absorbed, None, None)
    mass = torch.empty(ncell, dtype=torch.float32, device="cuda")
    S.skirt_dust_mass(grid.h, mass)
    feat = torch.empty((ncell, 32), dtype=torch.float32, device="cuda")
    tot = torch.empty(ncell, dtype=torch.float64, device="cuda")
    lam = np.ascontiguousarray(prob.wl.lam)
    S.skirt_band_features(absorbed, ncell, nl, lam, mass, feat, tot)
    exact = torch.empty((ncell, 100), dtype=torch.float64, device="cuda")
    S.skirt_dust_emission(absorbed, ncell, nl, lam, mass, S.EMIT_EXACT, None, exact)
    live = torch.nonzero((tot > 0) & (mass > 0)).flatten()
    assert live.numel() > 1_000_000
    # energy: every heated row sums to its absorbed power
    rel = ((exact.index_select(0, live).sum(dim=1) - tot.index_select(0, live)).abs() / tot.index_select(0, live))
    assert float(rel.max()) < 1e-12
    # sampled cells against the oracle
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    pick = live[torch.randperm(live.numel(), device="cuda", generator=gen)[:2000]]
    a_s = absorbed.index_select(0, pick).cpu().numpy()
    m_s = mass.index_select(0, pick).cpu().numpy().astype(np.float64)
    _, x_ref, t_ref = E.band_features(a_s, lam, m_s)
    np.testing.assert_allclose(tot.index_select(0, pick).cpu().numpy(), t_ref, rtol=1e-13)
    np.testing.assert_allclose(feat.index_select(0, pick).cpu().numpy(), x_ref, rtol=3e-7, atol=1e-6)
    e_ref, _, _ = E.exact_emission(a_s, lam, m_s)
    g = exact.index_select(0, pick).cpu().numpy()
    big = e_ref > 1e-9 * e_ref.sum(axis=1, keepdims=True)
    np.testing.assert_allclose(g[big], e_ref[big], rtol=1e-9)
    # the surrogate on every cell
    tr = live[torch.randperm(live.numel(), device="cuda", generator=gen)[:1_000_000]]
    net = S.MLP(seed=6)
    net.train(feat.index_select(0, tr).contiguous(), exact.index_select(0, tr).contiguous(), tr.numel())
    sur = torch.empty_like(exact)
    st = S.skirt_dust_emission(absorbed, ncell, nl, lam, mass, S.EMIT_SURROGATE, net, sur)
    net.close()
    grid.close()
    assert st["n_cells"] == ncell
    rs = (sur.index_select(0, live).sum(dim=1) - tot.index_select(0, live)).abs() / tot.index_select(0, live)
    assert float(rs.max()) < 1e-5
    e = (torch.linalg.vector_norm(sur.index_select(0, live) - exact.index_select(0, live), dim=1) /
         torch.linalg.vector_norm(exact.index_select(0, live), dim=1)).cpu().numpy()
    print("surrogate error over the heated cells: median", np.median(e), "p99", np.percentile(e, 99), "max", e.max(),
          "fallback", st["n_fallback"], "within 2%", (e <= 0.02).mean())
    assert st["n_fallback"] > 0
    assert np.median(e) < 0.005 and np.percentile(e, 99) < 0.01, (np.median(e), np.percentile(e, 99))
    assert (e > 0.02).sum() <= 10 and e.max() < 0.03, ((e > 0.02).sum(), e.max())
