"""The statistical parity criteria (tests/parity.py) on synthetic Monte Carlo
tallies, without a GPU: two independent samples of one process pass, a
sample of a process biased by 1% fails; the image rebinning bound and the
clumpy-medium split tolerance follow their formulas."""
import numpy as np
import pytest

import parity as P
from paper_1705_04702_gb300 import workloads as W


def _samples(rng, n_packets, n_cells, bias=0.0):
    """Per-packet tallies: each packet deposits an exponential amount in a few
    random cells; returns (per-packet contributions [n, cells])."""
    out = np.zeros((n_packets, n_cells))
    for p in range(n_packets):
        cells = rng.integers(0, n_cells, size=3)
        out[p, cells] += rng.exponential(1.0 + bias, size=3)
    return out


def test_split_check_accepts_independent_samples_and_rejects_a_bias():
    rng = np.random.default_rng(1)
    n_cells = 40
    matched = _samples(rng, 20000, n_cells)              # identical on both sides
    g_un = _samples(rng, 10000, n_cells)                 # unmatched: independent samples
    o_un = _samples(rng, 10000, n_cells)
    tot_g = matched.sum(0) + g_un.sum(0)
    tot_o = matched.sum(0) + o_un.sum(0)
    P.split_check(tot_g, tot_o, g_un.sum(0), o_un.sum(0), (g_un ** 2).sum(0), (o_un ** 2).sum(0), 1e-4, 1e-4)
    # a 10% bias of the unmatched packets' deposits: 3000 against K sigma = 5 x 346 over 10000 packets
    g_b = _samples(rng, 10000, n_cells, bias=0.1)
    with pytest.raises(AssertionError):
        P.split_check(matched.sum(0) + g_b.sum(0), tot_o, g_b.sum(0), o_un.sum(0), (g_b ** 2).sum(0),
                      (o_un ** 2).sum(0), 1e-4, 1e-4)
    # a 1e-3 error of the matched part fails the deterministic 1e-4 bar
    with pytest.raises(AssertionError):
        P.split_check(tot_g + 1e-3 * matched.sum(0), tot_o, g_un.sum(0), o_un.sum(0), (g_un ** 2).sum(0),
                      (o_un ** 2).sum(0), 1e-4, 1e-4)


def test_compare_tally_mc_allowance():
    rng = np.random.default_rng(2)
    ref = 1000.0 + rng.random(50)
    var = np.full(50, 4.0)                               # sigma 2 per entry
    allow = P.K_SIGMA * np.sqrt(2 * P.U_MAX * var)       # 0.447
    P.compare_tally_mc(ref + 0.9 * allow, ref, var, 1e-4, 0.0)
    with pytest.raises(AssertionError):
        P.compare_tally_mc(ref + 1e-4 * ref + 1.1 * allow, ref, var, 1e-4, 0.0)


def test_scattering_count_homogeneity():
    rng = np.random.default_rng(3)
    prob = W.sphere_problem(4000)
    prob = prob.with_packets(4000)
    rec = np.zeros((1, 4000, 8))
    same = rec.copy()
    same[0, :, 0] = rng.poisson(4.0, 4000)
    other = same.copy()
    other[0, :, 0] = rng.poisson(4.0, 4000)               # another sample of the same law
    assert P.scattering_counts_agree(same, other, prob) > P.CHI2_P_MIN
    shifted = same.copy()
    shifted[0, :, 0] = rng.poisson(4.4, 4000)             # 10% more scatterings
    with pytest.raises(AssertionError):
        P.scattering_counts_agree(shifted, other, prob)


def test_rebin_and_its_factor():
    img = np.arange(5 * 5, dtype=float).reshape(5, 5, 1)
    r = P.rebin(img, 2)
    assert r.shape == (3, 3, 1) and r.sum() == img.sum()
    assert r[2, 2, 0] == img[4, 4, 0] and r[0, 0, 0] == img[:2, :2, 0].sum()
    # disk images: |x|max 24, 512 pixels over 48 -> delta = 24 * 2^-21, smallest b with
    # 4 delta / (b dpx) <= 2.5e-5 is 32
    prob = W.disk_problem(10, n=16, npx=512)
    assert P.rebin_factor(prob, prob.instruments[0]) == 32
    # torus 48^2 over 2 (|x|max 1): b = 2
    prob = W.torus_problem(n=16, nlambda=2, packet_scale=1e-5, npx=48)
    assert P.rebin_factor(prob, prob.instruments[0]) == 2


def test_cell_split_rel():
    prob = W.torus_problem(n=48, nlambda=2, packet_scale=1e-5, npx=48)
    assert P.cell_split_rel(prob) == pytest.approx(1e-4 * (2.0 / 48) / (2 * 2.0))
