"""Comparison helpers for GPU-vs-oracle parity (shared by the GPU tests).

Tolerances (each derived in the design notes, section "Parity and
tolerances"):
* FP64 form: the GPU replays the oracle's packet histories with the same
  Philox streams; the only differences are rounding order (atomic
  accumulation order, exp/log implementations, reciprocal instead of
  division).  Per-packet records (fields scaled by the packet's launch
  luminosity, positions by the grid extent) and tallies agree to 1e-9.
* Mixed form, smooth media: FP32 traversal with ~2^-24 relative error per
  crossing.  At least 99.9% of the packets take the same number of
  scatterings with every record field within 1e-5 of its scale; tallies:
  L1-normalised difference below 1e-4 and every cell holding at least
  MIXED_CELL_SIGNIFICANT of the total within 1e-4.  Below that share a
  cell's tally is made of too few crossings to average the FP32 segment
  errors (absolute ~ t 2^-23 per crossing, t the distance from the
  traversal's start).
* Images: pixel indices are decided by FP32 positions, so a peel-off within
  ~|x| 2^-21 of a pixel border can land in the neighbouring pixel.  Images
  are compared element by element after summing b x b pixel blocks, with b
  the smallest power of two for which the share of a block's flux that can
  cross its border stays below a quarter of the tally tolerance
  (rebin_factor()).
* Clumpy media (100x density contrast): a path that grazes a clump boundary
  moves the next interaction point by up to the contrast times the
  perturbation, so FP32 rounding can make a history diverge from the
  oracle's (different interaction cells, then different scatterings).  Such
  a packet is a different Monte Carlo sample of the same process.  The
  criterion splits the packets: those whose records match within 1e-5 must
  give tallies within 1e-4 (the smooth-media bar), while the difference the
  others make, entry by entry, must stay within K_SIGMA standard deviations
  of the difference of two independent samples, sqrt(sum_p g_p^2 + o_p^2)
  over those packets' own single-packet tallies (split_check()); the
  distribution of the number of scatterings must be the oracle's
  (chi-square homogeneity, scattering_counts_agree()).
"""
import math

import numpy as np

REL_FP64 = 1e-9
REL_MIXED_PACKET = 1e-5
REL_MIXED_TALLY = 1e-4
MIXED_CELL_SIGNIFICANT = 1e-4
K_SIGMA = 5.0          # standard deviations allowed to the unmatched packets' tally difference
CHI2_P_MIN = 1e-4      # smallest accepted p-value of the scattering-count homogeneity test


def rel_err(a, b, floor):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def record_scales(prob):
    """Per-wavelength scales of the record fields: the packet's launch
    luminosity L0 for escaped/absorbed/residual, L0 times the summed
    peel-off normalisation 1/(4 pi d^2) for the peeled flux, the grid extent
    for the position."""
    import math
    L0 = np.where(prob.npk > 0, prob.wl.lsrc / np.maximum(prob.npk, 1).astype(np.float64), 0.0)
    norm = sum(1.0 / (4 * math.pi * i.distance ** 2) for i in prob.instruments)
    b = prob.grid.bbox
    extent = max(b[1] - b[0], b[3] - b[2], b[5] - b[4])
    return L0, norm, extent


def compare_records(gpu, ref, prob, rel, min_match=1.0, same_n_min=None):
    """gpu, ref: [nlambda, nrec, 8] records of the same packets.  A packet
    matches when it took the same number of scatterings and every other field
    agrees within rel of its scale (record_scales).  Returns the matching
    fraction over packets that exist; asserts it is >= min_match, and that
    the fraction with the same number of scatterings is >= same_n_min."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    L0, norm, extent = record_scales(prob)
    nrec = gpu.shape[1]
    exists = np.arange(nrec)[None, :] < prob.npk[:, None]
    scale = np.empty(gpu.shape[:2] + (7,))
    scale[..., 0:3] = L0[:, None, None]
    scale[..., 3] = (L0 * max(norm, 1e-300))[:, None]
    scale[..., 4:7] = extent
    err = np.abs(gpu[..., 1:] - ref[..., 1:]) / np.maximum(scale, 1e-300)
    ok = (gpu[..., 0] == ref[..., 0]) & np.all(err <= rel, axis=-1)
    ok = ok[exists]
    frac = ok.mean() if ok.size else 1.0
    if same_n_min is not None and ok.size:
        same = (gpu[..., 0] == ref[..., 0])[exists].mean()
        assert same >= same_n_min, ("scattering counts", same)
    bad = np.argwhere(exists & ~((gpu[..., 0] == ref[..., 0]) & np.all(err <= rel, axis=-1)))
    assert frac >= min_match, (frac, bad[:10], gpu[tuple(bad[:3].T)], ref[tuple(bad[:3].T)])
    return frac


def compare_tally(gpu, ref, rel, significant=1e-6, l1=None):
    """Element-wise relative check for entries holding >= significant of the
    total, and an L1-normalised bound over all entries."""
    gpu = np.asarray(gpu, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    tot = np.abs(ref).sum()
    if tot == 0:
        assert np.abs(gpu).sum() == 0
        return 0.0
    big = np.abs(ref) >= significant * tot
    e = rel_err(gpu[big], ref[big], 1e-300)
    assert e.size == 0 or e.max() <= rel, (e.max(), np.argmax(e))
    l1n = np.abs(gpu - ref).sum() / tot
    assert l1n <= (rel if l1 is None else l1), l1n
    return l1n


def position_error(prob):
    """Bound on the FP32 error of a peel-off's projected position: a few FP32
    roundings (the double-float position, the projection's products and
    sums) at the largest coordinate of the grid, |x|max 2^-21."""
    x0, x1, y0, y1, z0, z1 = prob.grid.bbox
    return max(abs(v) for v in (x0, x1, y0, y1, z0, z1)) * 2.0 ** -21


def rebin_factor(prob, ins, rel=REL_MIXED_TALLY):
    """Smallest power of two b (at most npx) such that a b x b block of
    pixels can lose or gain at most rel/4 of its flux across its border:
    the peel-offs within delta = position_error() of the block's four edges
    carry a share <= 4 delta / (b dpx) of a uniformly lit block's flux."""
    delta = position_error(prob)
    dpx = ins.fov / ins.npx
    b = 1
    while b < ins.npx and 4 * delta / (b * dpx) > rel / 4:
        b *= 2
    return b


def rebin(img, b):
    """Sums b x b pixel blocks of img [npx, npx, ...] (a ragged last block
    sums what is there)."""
    img = np.asarray(img)
    n = img.shape[0]
    m = -(-n // b)
    pad = np.zeros((m * b, m * b) + img.shape[2:], dtype=img.dtype)
    pad[:n, :n] = img
    return pad.reshape((m, b, m, b) + img.shape[2:]).sum(axis=(1, 3))


def compare_images(gpu_images, ref_images, prob, rel, significant):
    """Element-wise check of every instrument's image after rebinning by
    rebin_factor(): blocks holding >= significant of the instrument's total
    within rel, and the L1-normalised difference within rel."""
    for q, ins in enumerate(prob.instruments):
        b = rebin_factor(prob, ins, rel)
        compare_tally(rebin(gpu_images[q], b), rebin(ref_images[q], b), rel, significant=significant)


U_MAX = 1e-3  # largest share of unmatched packets the smooth-media record criterion allows


def compare_tally_mc(gpu, ref, var, rel, significant, u=U_MAX, k=K_SIGMA):
    """Tallies of many packets where the unmatched packets (a share u of all,
    at most U_MAX in smooth media) cannot be split off one by one: each entry
    holding >= significant of the total must agree within rel of its value
    plus k standard deviations of the difference that u of the packets make
    as independent samples, sqrt(2 u var) (var: the Monte Carlo variance of
    the entry's total, e.g. batch means); the L1-normalised difference within
    rel plus the same allowance summed.  Returns the L1 difference."""
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    var = np.asarray(var, np.float64).ravel()
    tot = np.abs(ref).sum()
    allow = k * np.sqrt(2.0 * u * var)
    big = np.abs(ref) >= significant * tot
    d = np.abs(gpu - ref)
    bad = big & (d > rel * np.abs(ref) + allow)
    assert not bad.any(), ("entries beyond rel + k sigma", int(bad.sum()), (d / np.abs(ref))[bad][:5],
                           (allow / np.abs(ref))[bad][:5])
    l1 = d.sum() / tot
    assert l1 <= rel + allow.sum() / tot, (l1, allow.sum() / tot)
    return float(l1)


def cell_split_rel(prob, rel=REL_MIXED_TALLY):
    """Record tolerance below which a packet's per-cell deposits agree within
    rel even in a cell that the packet alone lights: a displacement delta of
    the packet's path moves its deposit boundaries by delta, which changes a
    crossing of length h/2 (h the smallest cell size) by 2 delta / h of its
    deposit; delta = rel h / 2, as a fraction of the grid extent (the record
    scale of positions)."""
    x0, x1, y0, y1, z0, z1 = prob.grid.bbox
    extent = max(x1 - x0, y1 - y0, z1 - z0)
    h = min((x1 - x0) / prob.grid.nx, (y1 - y0) / prob.grid.ny, (z1 - z0) / prob.grid.nz)
    return min(REL_MIXED_PACKET, rel * h / (2.0 * extent))


def unmatched(gpu, ref, prob, rel):
    """Boolean [nlambda, nrec]: packets that exist and whose records differ
    (another number of scatterings, or a field beyond rel of its scale)."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    L0, norm, extent = record_scales(prob)
    nrec = gpu.shape[1]
    exists = np.arange(nrec)[None, :] < prob.npk[:, None]
    scale = np.empty(gpu.shape[:2] + (7,))
    scale[..., 0:3] = L0[:, None, None]
    scale[..., 3] = (L0 * max(norm, 1e-300))[:, None]
    scale[..., 4:7] = extent
    err = np.abs(gpu[..., 1:] - ref[..., 1:]) / np.maximum(scale, 1e-300)
    ok = (gpu[..., 0] == ref[..., 0]) & np.all(err <= rel, axis=-1)
    return exists & ~ok


def single_packet_problem(prob, j):
    """The problem restricted to wavelength j (its packet count, hence its
    packet luminosity, unchanged)."""
    npk = np.zeros_like(prob.npk)
    npk[j] = prob.npk[j]
    return prob.with_packets(npk)


def _parts(absorbed, sed, images, bins):
    return {"absorbed": np.asarray(absorbed, np.float64), "sed": np.asarray(sed, np.float64),
            "images": [rebin(im, b) for im, b in zip(images, bins)]}


def _zero_like(parts):
    return {"absorbed": np.zeros_like(parts["absorbed"]), "sed": np.zeros_like(parts["sed"]),
            "images": [np.zeros_like(im) for im in parts["images"]]}


def _add(acc, parts, power):
    acc["absorbed"] += parts["absorbed"] ** power
    acc["sed"] += parts["sed"] ** power
    for q, im in enumerate(parts["images"]):
        acc["images"][q] += im ** power


def packet_tallies_oracle(oracle_lib, prob, pairs, bins, template, **trace_kw):
    """Sums and sums of squares, over the packets (j, i) in pairs, of each
    packet's own tallies from the oracle (images rebinned by bins[q])."""
    acc, sq = _zero_like(template), _zero_like(template)
    for j, i in pairs:
        r = oracle_lib.trace(single_packet_problem(prob, int(j)), int(i), int(i) + 1, **trace_kw)
        parts = _parts(r["absorbed"], r["sed"], r["images"], bins)
        _add(acc, parts, 1)
        _add(sq, parts, 2)
    return acc, sq


def packet_tallies_gpu(S, grid, prob, pairs, bins, template, precision, **run_kw):
    """As packet_tallies_oracle, from single-packet GPU calls (packet i of
    wavelength j through first_packet / total_packets)."""
    acc, sq = _zero_like(template), _zero_like(template)
    n = prob.wl.n
    for j, i in pairs:
        one = np.zeros(n, dtype=np.uint64)
        one[j] = 1
        first = np.zeros(n, dtype=np.uint64)
        first[j] = i
        g = S.run_problem(prob.with_packets(one), grid, precision=precision, first_packet=first,
                          total_packets=prob.npk, **run_kw)
        parts = _parts(g["absorbed"].cpu().numpy(), g["sed"].cpu().numpy()[:len(prob.instruments)],
                       [im.cpu().numpy() for im in g["images"]], bins)
        _add(acc, parts, 1)
        _add(sq, parts, 2)
    return acc, sq


# The mixed form ends a deposit or peel-off traversal once its optical depth
# passes 30 and drops contributions below the FP32 range (design reading
# 11): a packet loses at most e^-30 of its luminosity per traversal, so an
# entry can differ by up to this share of the luminosity of the packets
# behind it, times the traversals of a packet (bounded here by 100).
CUT_SHARE = 100 * math.exp(-30.0)


def split_check(gpu_tot, ref_tot, gpu_f, ref_f, gpu_f2, ref_f2, rel, significant, k=K_SIGMA, atol=0.0):
    """gpu_tot / ref_tot: tallies of all packets; gpu_f / ref_f: the sums of
    the unmatched packets' own tallies, gpu_f2 / ref_f2 their sums of
    squares.  The matched packets' part (total minus unmatched) must agree
    within rel (entries >= significant of the total, and L1); the unmatched
    part must differ by at most k standard deviations of the difference of two
    independent samples of those packets, sqrt(gpu_f2 + ref_f2), entry by
    entry and summed over all entries, plus atol (the optical-depth cut-off's
    share of those packets' luminosity, CUT_SHARE).  Returns (matched part's
    L1, unmatched part's L1 share of the total)."""
    g = np.asarray(gpu_tot, np.float64).ravel()
    r = np.asarray(ref_tot, np.float64).ravel()
    gf = np.asarray(gpu_f, np.float64).ravel()
    rf = np.asarray(ref_f, np.float64).ravel()
    var = np.asarray(gpu_f2, np.float64).ravel() + np.asarray(ref_f2, np.float64).ravel()
    # the subtraction leaves FP64 rounding of the totals, far below rel
    l1 = compare_tally(g - gf, r - rf, rel, significant=significant)
    d = gf - rf
    sig = np.sqrt(var)
    bad = np.abs(d) > k * sig + 1e-12 * np.abs(r) + atol
    assert not bad.any(), ("unmatched packets beyond k sigma", int(bad.sum()), d[bad][:5], sig[bad][:5])
    assert abs(d.sum()) <= k * np.sqrt(var.sum()) + 1e-12 * abs(r.sum()) + atol * d.size, (d.sum(),
                                                                                          np.sqrt(var.sum()))
    return l1, float(np.abs(d).sum() / max(np.abs(r).sum(), 1e-300))


def check_mixed(S, oracle_lib, grid, prob, g, r, chaotic=False, min_match=0.999,
                significant=MIXED_CELL_SIGNIFICANT, gpu_kw=None, oracle_kw=None):
    """The mixed form's run g against the oracle's run r of the same packets
    (records of every packet).  Records: smooth media need min_match of the
    packets to match (same scatterings, fields within 1e-5); in a clumpy
    medium the scattering-count distributions must agree instead.  Tallies:
    the unmatched packets' single-packet tallies are taken from both sides;
    the rest (absorbed table, SEDs, rebinned images, ledger) must agree within
    1e-4 and the unmatched part within K_SIGMA (split_check,
    record_sigma_check).  In smooth media a packet is matched within 1e-5
    (significant cells average many packets); in a clumpy medium, where a
    significant cell can be lit by one or two packets whose paths drift, within
    cell_split_rel().  Returns a summary."""
    gr = g["records"].cpu().numpy()
    rr = r["records"]
    assert gr.shape[1] >= int(prob.npk.max()), "records of every packet are needed"
    out = {}
    if chaotic:
        out["chi2_p"] = scattering_counts_agree(gr, rr, prob)
    else:
        out["matched"] = compare_records(gr, rr, prob, REL_MIXED_PACKET, min_match, same_n_min=0.999)
    um = unmatched(gr, rr, prob, cell_split_rel(prob) if chaotic else REL_MIXED_PACKET)
    out["unmatched"] = int(um.sum())
    record_sigma_check(gr, rr, prob, um)
    gpu_kw = gpu_kw or {}
    oracle_kw = oracle_kw or {}
    bins = [rebin_factor(prob, ins) for ins in prob.instruments]
    template = _parts(r["absorbed"], r["sed"], r["images"], bins)
    pairs = np.argwhere(um)
    L0, _, _ = record_scales(prob)
    cut = CUT_SHARE * float(sum(L0[j] for j, _ in pairs))  # the unmatched packets' luminosity
    gf, gf2 = packet_tallies_gpu(S, grid, prob, pairs, bins, template, S.PREC_MIXED, **gpu_kw)
    of, of2 = packet_tallies_oracle(oracle_lib, prob, pairs, bins, template, **oracle_kw)
    out["absorbed"] = split_check(g["absorbed"].cpu().numpy(), r["absorbed"], gf["absorbed"], of["absorbed"],
                                  gf2["absorbed"], of2["absorbed"], REL_MIXED_TALLY, significant, atol=cut)
    if prob.instruments:
        out["sed"] = split_check(g["sed"].cpu().numpy(), r["sed"], gf["sed"], of["sed"], gf2["sed"], of2["sed"],
                                 REL_MIXED_TALLY, 0.0, atol=cut)
        for q in range(len(prob.instruments)):
            gi = rebin(g["images"][q].cpu().numpy(), bins[q])
            ri = rebin(r["images"][q], bins[q])
            out[f"image{q}"] = split_check(gi, ri, gf["images"][q], of["images"][q], gf2["images"][q],
                                           of2["images"][q], REL_MIXED_TALLY, significant, atol=cut)
    # the ledger per wavelength: emitted, absorbed, escaped, residual; the
    # unmatched packets' shares come from their records
    um_g = np.stack([np.where(um, gr[..., f], 0.0).sum(axis=1) for f in (2, 1, 3)], axis=1)
    um_r = np.stack([np.where(um, rr[..., f], 0.0).sum(axis=1) for f in (2, 1, 3)], axis=1)
    lg = np.asarray(g["ledger_per_lambda"])
    lr = np.asarray(r["ledger"])
    np.testing.assert_allclose(lg[:, 0], lr[:, 0], rtol=REL_MIXED_TALLY, atol=1e-300)
    np.testing.assert_allclose(lg[:, 1:] - um_g, lr[:, 1:] - um_r, rtol=REL_MIXED_TALLY,
                               atol=1e-12 * float(lr[:, 0].max()))
    return out


def scattering_counts_agree(gpu, ref, prob, p_min=CHI2_P_MIN):
    """Chi-square test of homogeneity between the GPU's and the oracle's
    numbers of scatterings over the sampled packets (bins pooled until every
    expected count is >= 5).  The two samples share their random streams,
    which makes them closer than independent samples, so the test is
    conservative.  Returns the p-value; asserts p >= p_min."""
    from scipy import stats
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    exists = np.arange(gpu.shape[1])[None, :] < prob.npk[:, None]
    a = gpu[..., 0][exists].astype(np.int64)
    b = ref[..., 0][exists].astype(np.int64)
    hi = int(max(a.max(), b.max())) + 1
    ca = np.bincount(a, minlength=hi).astype(np.float64)
    cb = np.bincount(b, minlength=hi).astype(np.float64)
    # pool neighbouring bins from the top down until each pooled bin has >= 10 packets in all
    rows, cur = [], np.zeros(2)
    for k in range(hi - 1, -1, -1):
        cur += (ca[k], cb[k])
        if cur.sum() >= 10:
            rows.append(cur.copy())
            cur[:] = 0
    if rows and cur.sum():
        rows[-1] += cur
    tab = np.array(rows)
    if tab.shape[0] < 2 or np.all(tab[:, 0] == tab[:, 1]):
        return 1.0
    p = stats.chi2_contingency(tab.T, correction=False)[1]
    assert p >= p_min, ("scattering-count distributions differ", p, tab.T)
    return float(p)


def record_sigma_check(gpu, ref, prob, mask, k=K_SIGMA):
    """For the record fields escaped, absorbed, residual and peeled flux (the
    packets' own shares of the ledger and of the SEDs): over the packets in
    mask, the summed GPU-minus-oracle difference per wavelength and over all
    wavelengths stays within k standard deviations of the difference of two
    independent samples (sqrt of the summed squares of both), plus the
    optical-depth cut-off's share (CUT_SHARE) of those packets' luminosity."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    L0, norm, _ = record_scales(prob)
    for f in (1, 2, 3, 4):
        g = np.where(mask, gpu[..., f], 0.0)
        r = np.where(mask, ref[..., f], 0.0)
        d = (g - r).sum(axis=1)
        sig = np.sqrt((g ** 2 + r ** 2).sum(axis=1))
        cut = CUT_SHARE * L0 * mask.sum(axis=1) * (norm if f == 4 else 1.0)
        assert np.all(np.abs(d) <= k * sig + cut + 1e-300), ("field", f, d, sig)
        assert abs(d.sum()) <= k * np.sqrt((sig ** 2).sum()) + cut.sum() + 1e-300, ("field", f, d.sum())
