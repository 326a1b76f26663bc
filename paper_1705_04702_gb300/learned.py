"""The learned form of the panchromatic run: stellar emission phase, dust
emission from the absorbed field through the MLP surrogate (exact
solver as fallback and as the reference the surrogate is scored against), and
the dust re-emission trace (arXiv:1705.04702 Sect. 3.2, stellar emission phase -> dust emission phase).

Every step runs in the library's kernels through the C ABI; this module only
allocates device memory, picks the training cells and times the stages.
"""
from __future__ import annotations

import time

import numpy as np

from . import skirt as S
from . import workloads as W


def _sync():
    import torch
    torch.cuda.synchronize()


def run_learned(n=256, nlambda=200, packet_scale=1.0, n_train=1_000_000, n_test=100_000, epochs=200, batch=2048,
                lr=2e-3, reemit_per_lambda=1_000_000, seed=1, compare_exact=True, autotune=False, keep=False):
    """Runs the learned form on the clumpy torus and returns a report: stage
    times [s], the surrogate's error against the exact solver on held-out
    cells (per-cell relative L2 over the 100 emission wavelengths), the
    fallback count, and the energy bookkeeping of both traces."""
    import torch
    rep = {"grid": n, "nlambda": nlambda}
    prob = W.torus_problem(n=n, nlambda=nlambda, seed=seed, packet_scale=packet_scale)
    grid = S.Grid(prob.grid)
    ncell, NL = grid.ncell, prob.wl.n
    lam = np.ascontiguousarray(prob.wl.lam)
    ins = S.make_instruments(prob.instruments)
    npix = sum(i.npx * i.npx for i in prob.instruments)
    dev = "cuda"

    # ---- stellar emission phase
    absorbed = torch.zeros((ncell, NL), dtype=torch.float64, device=dev)
    images = torch.zeros(npix * NL, dtype=torch.float64, device=dev)
    sed = torch.zeros((len(ins), NL), dtype=torch.float64, device=dev)
    opts = S.skirt_trace_opts_default()
    opts.use_graph = 1
    tables = S.Tables(prob.wl)
    src = S.make_source(prob.source)
    if autotune:
        S.skirt_autotune(grid.h, src, tables.c, prob.npk, prob.seed, ins, opts, 0.01, absorbed, images, sed)
    _sync()
    t0 = time.perf_counter()
    _, led, _ = S.skirt_trace(grid.h, src, tables.c, prob.npk, prob.seed, ins, opts, absorbed, images, sed)
    _sync()
    rep["t_stellar_trace"] = time.perf_counter() - t0
    rep["stellar_packets"] = prob.total_packets
    rep["stellar_ledger"] = led

    # ---- dust masses, band features of every cell
    mass = torch.empty(ncell, dtype=torch.float32, device=dev)
    S.skirt_dust_mass(grid.h, mass)
    feat = torch.empty((ncell, S.NBANDS), dtype=torch.float32, device=dev)
    tot = torch.empty(ncell, dtype=torch.float64, device=dev)
    S.skirt_band_features(absorbed, ncell, NL, lam, mass, feat, tot)

    # ---- training set: exact solutions for a random sample of heated dusty cells
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    live = torch.nonzero((tot > 0) & (mass > 0)).flatten()
    n_train = int(min(n_train, max(len(live) - n_test, len(live) // 2)))
    n_test = int(min(n_test, len(live) - n_train))
    pick = live[torch.randperm(len(live), device=dev, generator=gen)[:n_train + n_test]]
    tr, te = pick[:n_train].contiguous(), pick[n_train:].contiguous()
    a_tr = absorbed.index_select(0, tr)
    m_tr = mass.index_select(0, tr)
    ex_tr = torch.empty((n_train, S.NEMIT), dtype=torch.float64, device=dev)
    _sync()
    t0 = time.perf_counter()
    S.skirt_dust_emission(a_tr, n_train, NL, lam, m_tr, S.EMIT_EXACT, None, ex_tr)
    _sync()
    rep["t_training_labels"] = time.perf_counter() - t0
    net = S.MLP(seed=seed)
    t0 = time.perf_counter()
    hist = net.train(feat.index_select(0, tr), ex_tr, n_train, epochs=epochs, batch=batch, lr=lr, seed=seed)
    _sync()
    rep["t_training"] = time.perf_counter() - t0
    rep["n_train"], rep["n_test"] = n_train, n_test
    rep["guard_share_max"] = net.get_guard()
    rep["loss_first_last"] = [float(hist[0]), float(hist[-1])]
    del a_tr, ex_tr

    # ---- dust emission of every cell: surrogate (with fallback), and exact
    em_s = torch.empty((ncell, S.NEMIT), dtype=torch.float64, device=dev)
    _sync()
    t0 = time.perf_counter()
    st_s = S.skirt_dust_emission(absorbed, ncell, NL, lam, mass, S.EMIT_SURROGATE, net, em_s)
    _sync()
    rep["t_emission_surrogate"] = time.perf_counter() - t0
    rep["surrogate_stats"] = st_s
    if compare_exact:
        em_e = torch.empty((ncell, S.NEMIT), dtype=torch.float64, device=dev)
        _sync()
        t0 = time.perf_counter()
        st_e = S.skirt_dust_emission(absorbed, ncell, NL, lam, mass, S.EMIT_EXACT, None, em_e)
        _sync()
        rep["t_emission_exact"] = time.perf_counter() - t0
        rep["exact_stats"] = st_e
        # error of the surrogate on held-out cells and on every heated cell
        def rel_l2(a, b):
            return torch.linalg.vector_norm(a - b, dim=1) / torch.linalg.vector_norm(b, dim=1).clamp_min(1e-300)
        e_te = rel_l2(em_s.index_select(0, te), em_e.index_select(0, te)).cpu().numpy()
        e_all = rel_l2(em_s.index_select(0, live), em_e.index_select(0, live)).cpu().numpy()
        rep["err_heldout"] = {p: float(np.percentile(e_te, p)) for p in (50, 90, 99)} | {"max": float(e_te.max())}
        rep["err_all_cells"] = {p: float(np.percentile(e_all, p)) for p in (50, 90, 99)} | {"max": float(e_all.max())}
        rep["frac_cells_within_2pct"] = float((e_all <= 0.02).mean())
        rep["energy_rel_err_surrogate"] = float(((em_s.sum(dim=1) - tot).abs().sum() / tot.sum()).item())
        del em_e
    rep["heated_cells"] = int(len(live))

    # ---- dust emission phase: re-emission trace from the surrogate's table
    lam_ir, _ = S.skirt_emission_grid()
    wl_ir = W.powerlaw_wavelengths(S.NEMIT, float(lam_ir[0]), float(lam_ir[-1]), alb_short=0.3, alb_long=0.0)
    wl_ir.lsrc = None  # the emission table's column sums
    npk_ir = np.full(S.NEMIT, int(reemit_per_lambda), dtype=np.uint64)
    src_d = S.make_source(W.Source(W.SRC_DUST), emission=em_s)
    t_ir = S.Tables(wl_ir)
    absorbed_d = torch.zeros((ncell, S.NEMIT), dtype=torch.float64, device=dev)
    images_d = torch.zeros(npix * S.NEMIT, dtype=torch.float64, device=dev)
    sed_d = torch.zeros((len(ins), S.NEMIT), dtype=torch.float64, device=dev)
    o2 = S.skirt_trace_opts_default()
    o2.phase = 1
    _sync()
    t0 = time.perf_counter()
    _, led_d, _ = S.skirt_trace(grid.h, src_d, t_ir.c, npk_ir, prob.seed, ins, o2, absorbed_d, images_d, sed_d)
    _sync()
    rep["t_reemission_trace"] = time.perf_counter() - t0
    rep["reemission_packets"] = int(npk_ir.sum())
    rep["reemission_ledger"] = led_d
    rep["emitted_dust_luminosity"] = float(em_s.sum().item())

    rep["t_run_surrogate"] = rep["t_stellar_trace"] + rep["t_emission_surrogate"] + rep["t_reemission_trace"]
    if compare_exact:
        rep["t_run_exact"] = rep["t_stellar_trace"] + rep["t_emission_exact"] + rep["t_reemission_trace"]
        rep["speedup_emission_step"] = rep["t_emission_exact"] / rep["t_emission_surrogate"]
        rep["speedup_whole_run"] = rep["t_run_exact"] / rep["t_run_surrogate"]
        rep["speedup_whole_run_incl_training"] = rep["t_run_exact"] / (
            rep["t_run_surrogate"] + rep["t_training"] + rep["t_training_labels"])
    if keep:
        rep["_tensors"] = {"absorbed": absorbed, "mass": mass, "em_s": em_s, "absorbed_d": absorbed_d, "sed_d": sed_d}
    net.close()
    grid.close()
    return rep
