"""Pins of the oracle's packet life cycle against closed forms, exact
quadratures with independent geometry, invariants and brute force."""
import math

import numpy as np
import pytest

from paper_1705_04702_gb300 import workloads as W


# ---------------------------------------------------------------------------
# independent exact geometry for the tests: ray / axis-aligned box
# intersection by the slab method, cell by cell
# ---------------------------------------------------------------------------
def _cell_intervals(grid, p, k):
    """For every cell, the parameter interval [t_in, t_out] (t >= 0) of the
    ray p + t k inside that cell (empty: t_in >= t_out)."""
    x0, x1, y0, y1, z0, z1 = grid.bbox
    n = (grid.nx, grid.ny, grid.nz)
    los = (x0, y0, z0)
    his = (x1, y1, z1)
    tin = np.zeros((grid.nz, grid.ny, grid.nx))
    tout = np.full((grid.nz, grid.ny, grid.nx), np.inf)
    for a in range(3):
        d = (his[a] - los[a]) / n[a]
        faces = los[a] + np.arange(n[a] + 1) * d
        if k[a] != 0:
            t1 = (faces[:-1] - p[a]) / k[a]
            t2 = (faces[1:] - p[a]) / k[a]
            lo_, hi_ = np.minimum(t1, t2), np.maximum(t1, t2)
        else:
            inside = (faces[:-1] <= p[a]) & (p[a] < faces[1:])
            lo_ = np.where(inside, -np.inf, np.inf)
            hi_ = np.where(inside, np.inf, -np.inf)
        shape = [1, 1, 1]
        shape[2 - a] = n[a]
        tin = np.maximum(tin, lo_.reshape(shape))
        tout = np.minimum(tout, hi_.reshape(shape))
    return tin.ravel(), tout.ravel()


def _tau_before_and_in(grid, kscale, p, k):
    tin, tout = _cell_intervals(grid, p, k)
    kr = grid.kr.astype(np.float64).ravel() * kscale
    ok = tout > tin
    tin, tout, kr_ok = tin[ok], tout[ok], kr[ok]
    order = np.argsort(tin)
    tau_in = kr_ok[order] * (tout[order] - tin[order])
    tau_before = np.concatenate([[0.0], np.cumsum(tau_in)[:-1]])
    cells = np.nonzero(ok)[0][order]
    return cells, tau_before, tau_in


# ---------------------------------------------------------------------------
def test_slab_beam_pure_absorber(oracle_lib):
    """Collimated beam through a face-aligned pure absorber: transmitted
    e^{-tau/mu}, and layer m absorbs e^{-tau_{m-1}/mu} - e^{-tau_m/mu}."""
    layer_tau = np.array([0.2, 0.3, 0.5, 4.0], dtype=np.float32).astype(np.float64)
    grid = W.slab_grid(layer_tau)
    for mu in (1.0, 0.6):
        k = (math.sqrt(1 - mu * mu), 0.0, mu)
        prob = W.beam_problem(grid, (0.1, 0.2, 0.0), k, npackets=1, albedo=0.0)
        r = oracle_lib.trace(prob, nrec=1)
        tau_total = layer_tau.sum() / mu
        rec = r["records"][0, 0]
        assert rec[1] == pytest.approx(math.exp(-tau_total), rel=1e-14)
        cum = np.concatenate([[0.0], np.cumsum(layer_tau)]) / mu
        expect = np.exp(-cum[:-1]) - np.exp(-cum[1:])
        # the beam stays in one (x,y) column; sum absorbed over x,y per layer
        got = r["absorbed"][:, 0].reshape(grid.nz, -1).sum(axis=1)
        np.testing.assert_allclose(got, expect, rtol=1e-13)
        assert rec[2] + rec[1] == pytest.approx(1.0, rel=1e-14)


def test_forced_interaction_is_truncated_exponential(oracle_lib):
    """With one allowed interaction the interaction optical depth of a beam
    through a uniform slab follows the exponential distribution truncated at
    the slab's optical depth: CDF (1 - e^{-tau}) / (1 - e^{-tau_path})."""
    grid = W.slab_grid(np.full(8, 0.25))  # tau_path = 2 along +z, 1/length per unit
    prob = W.beam_problem(grid, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), npackets=4000, albedo=0.5)
    prob.max_events = 1
    r = oracle_lib.trace(prob, nrec=4000)
    assert r["status"] & oracle_lib.ERR_EVENT_CAP
    tau_int = r["records"][0, :, 7] * 0.25  # z of the interaction times kappa*rho
    F = np.sort((1 - np.exp(-tau_int)) / (1 - np.exp(-2.0)))
    ks = np.max(np.abs(F - (np.arange(1, F.size + 1) - 0.5) / F.size))
    assert ks < 1.63 / math.sqrt(F.size)  # 1% Kolmogorov-Smirnov level


def test_cube_escape_per_packet(oracle_lib):
    """Point source at the centre of a uniform cube (kr=1, half-width 1, the
    source on a corner shared by 8 cells), pure absorber: each packet escapes
    with e^{-1/max|k_a|}, k its launch direction, which equals the direction
    of its interaction point."""
    grid = W.uniform_grid(16, half=1.0, kr=1.0)
    prob = W.Problem("cube", grid, W.Source(W.SRC_POINT, (0.0, 0.0, 0.0)),
                     W.single_wavelength(albedo=0.0, g=0.0), np.array([3000], np.uint64),
                     [W.Instrument(100.0, 0.0, 0.0, 2.0, 16)])
    r = oracle_lib.trace(prob, nrec=3000)
    rec = r["records"][0]
    L0 = 1.0 / 3000
    pos = rec[:, 5:8]
    k = pos / np.linalg.norm(pos, axis=1, keepdims=True)
    np.testing.assert_allclose(rec[:, 1], L0 * np.exp(-1.0 / np.abs(k).max(axis=1)), rtol=1e-10)
    # the mean over packets agrees with the quadrature over the sphere of
    # e^{-1/max|k_a|} (midpoint rule in mu and phi)
    nmu, nphi = 1200, 2400
    mu = -1 + (np.arange(nmu) + 0.5) * 2 / nmu
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    st = np.sqrt(1 - mu * mu)[:, None]
    kmax = np.maximum(np.maximum(np.abs(st * np.cos(phi)), np.abs(st * np.sin(phi))), np.abs(mu)[:, None])
    vals = np.exp(-1 / kmax)
    mean, sd = vals.mean(), vals.std()
    esc = rec[:, 1].sum()
    assert abs(esc - mean) < 4 * sd / math.sqrt(3000)


def test_sphere_escape_against_exact_voxel_geometry(oracle_lib):
    """Point source in the 32^3 voxelised uniform sphere (tau_R = 1), pure
    absorber: per-packet escape equals e^{-tau(k)}, tau(k) from the slab-method
    intersection with every cell; the mean approaches e^{-1} for the smooth
    sphere within the voxelisation error."""
    prob = W.sphere_problem(npackets=20000, albedo=0.0)
    r = oracle_lib.trace(prob, nrec=300)
    rec = r["records"][0]
    L0 = 1.0 / 20000
    for q in range(0, 300, 3):
        kdir = rec[q, 5:8] / np.linalg.norm(rec[q, 5:8])
        _, tb, ti = _tau_before_and_in(prob.grid, 1.0, np.zeros(3), kdir)
        assert rec[q, 1] == pytest.approx(L0 * math.exp(-(tb[-1] + ti[-1])), rel=1e-9)
    frac = r["ledger"][0, 2]
    assert frac == pytest.approx(math.exp(-1.0), rel=0.02)


@pytest.mark.parametrize("src", [(0.13, -0.27, 0.31), (0.0, 0.0, 0.0)])
def test_two_cube_grid_brute_force(oracle_lib, src):
    """2^3 grid with eight different densities, point source (off-centre, and
    on the corner shared by all eight cells), pure absorber.  The expected
    fraction absorbed in each cell, the direction average of
    e^{-tau_before}(1 - e^{-tau_in}), is computed by quadrature with exact
    ray/box intersections; the Monte Carlo tally must agree within 4 sigma."""
    kr = np.array([0.3, 1.1, 0.05, 2.0, 0.7, 0.0, 1.6, 0.45], dtype=np.float32).reshape(2, 2, 2)
    grid = W.Grid(2, 2, 2, (-1.0, 1.0, -1.0, 1.0, -1.0, 1.0), kr)
    N = 40000
    prob = W.Problem("two", grid, W.Source(W.SRC_POINT, src), W.single_wavelength(albedo=0.0),
                     np.array([N], np.uint64), [])
    r = oracle_lib.trace(prob)
    got = r["absorbed"][:, 0]
    nmu, nphi = 240, 480
    acc = np.zeros(8)
    acc2 = np.zeros(8)
    for mu in -1 + (np.arange(nmu) + 0.5) * 2 / nmu:
        st = math.sqrt(1 - mu * mu)
        for phi in (np.arange(nphi) + 0.5) * 2 * math.pi / nphi:
            k = np.array([st * math.cos(phi), st * math.sin(phi), mu])
            cells, tb, ti = _tau_before_and_in(grid, 1.0, np.asarray(src, float), k)
            f = np.zeros(8)
            f[cells] = np.exp(-tb) * (-np.expm1(-ti))
            acc += f
            acc2 += f * f
    M = nmu * nphi
    mean = acc / M
    sd = np.sqrt(np.maximum(acc2 / M - mean ** 2, 0))
    assert np.all(np.abs(got - mean) <= 4 * sd / math.sqrt(N) + 1e-4)
    assert got[5] == 0.0  # the empty cell absorbs nothing


def test_optically_thin_peel_off_flux_and_pixel(oracle_lib):
    """tau -> 0: every packet's emission peel-off carries L/(4 pi d^2) into
    the pixel under the source.  Face-on (inclination 0, azimuth 0) the image
    columns run along +y and the rows along -x; edge-on (inclination 90) the
    rows run along +z."""
    grid = W.uniform_grid(8, kr=1e-9)
    src = (0.33, -0.17, 0.46)
    ins = [W.Instrument(50.0, 0.0, 0.0, 2.0, 20), W.Instrument(50.0, 90.0, 0.0, 2.0, 20)]
    N = 500
    prob = W.Problem("thin", grid, W.Source(W.SRC_POINT, src), W.single_wavelength(albedo=0.5),
                     np.array([N], np.uint64), ins)
    r = oracle_lib.trace(prob)
    F = 1.0 / (4 * math.pi * 50.0 ** 2)
    for q in range(2):
        assert r["sed"][q, 0] == pytest.approx(F, rel=1e-6)
        assert r["images"][q].sum() == pytest.approx(F, rel=1e-6)
    # pixel size 0.1: face-on column from y=-0.17 -> 8, row from -x=-0.33 -> 6
    assert r["images"][0][6, 8, 0] == pytest.approx(F, rel=1e-6)
    # edge-on (observer on +x): column from y -> 8, row from z=0.46 -> 14
    assert r["images"][1][14, 8, 0] == pytest.approx(F, rel=1e-6)


def test_thin_sphere_scattered_light_normalisation(oracle_lib):
    """Optically thin sphere (tau_R = 0.01), central source: the first
    scattering peel-off carries on average L albedo (1 - e^{-tau_R}) / (4 pi d^2)
    because the HG phase function averages to 1 over isotropic incidence."""
    grid = W.sphere_grid(16, kr_in=0.01)
    N = 60000
    albedo = 0.5
    prob = W.Problem("thin_sphere", grid, W.Source(W.SRC_POINT, (0.0, 0.0, 0.0)),
                     W.single_wavelength(albedo=albedo, g=0.6), np.array([N], np.uint64),
                     [W.Instrument(100.0, 30.0, 0.0, 2.0, 16)])
    r = oracle_lib.trace(prob)
    F = 1.0 / (4 * math.pi * 100.0 ** 2)
    # every emission peel-off leaves the centre along the same line of sight
    inc = math.radians(30.0)
    kobs = np.array([math.sin(inc), 0.0, math.cos(inc)])
    _, tb, ti = _tau_before_and_in(grid, 1.0, np.zeros(3), kobs)
    emission_part = math.exp(-(tb[-1] + ti[-1]))
    scat = r["sed"][0, 0] / F - emission_part
    tau = 0.01
    expect = albedo * (1 - math.exp(-tau))
    assert scat == pytest.approx(expect, rel=0.04)


@pytest.mark.parametrize("maker", ["sphere", "disk", "torus"])
def test_energy_conservation_per_packet(oracle_lib, maker):
    """emitted = absorbed + escaped + residual for every packet, to FP64
    rounding, and for the wavelength totals (compensated sums)."""
    if maker == "sphere":
        prob = W.sphere_problem(3000)
    elif maker == "disk":
        prob = W.disk_problem(300, n=64, nlambda=3, npx=32)
    else:
        prob = W.torus_problem(n=32, nlambda=6, packet_scale=2e-4, npx=16)
    nrec = int(prob.npk.max())
    r = oracle_lib.trace(prob, nrec=nrec)
    assert r["status"] == 0
    for lam in range(prob.wl.n):
        n = int(prob.npk[lam])
        if n == 0:
            continue
        L0 = prob.wl.lsrc[lam] / n
        rec = r["records"][lam, :n]
        closure = (L0 - rec[:, 1] - rec[:, 2] - rec[:, 3]) / L0
        assert np.max(np.abs(closure)) < 1e-13
        tot = math.fsum(rec[:, 1]) + math.fsum(rec[:, 2]) + math.fsum(rec[:, 3])
        assert tot == pytest.approx(prob.wl.lsrc[lam], rel=1e-12)
        assert r["ledger"][lam, 0] == pytest.approx(prob.wl.lsrc[lam], rel=1e-12)
        # the absorbed table holds exactly what the packets deposited
        assert math.fsum(r["absorbed"][:, lam]) == pytest.approx(math.fsum(rec[:, 2]), rel=1e-12)


def test_packet_ranges_compose(oracle_lib):
    """Counter-based random numbers: running packets [0,N) equals running
    [0,N/2) and [N/2,N) separately and adding the tallies."""
    prob = W.sphere_problem(2000)
    a = oracle_lib.trace(prob)
    b = oracle_lib.trace(prob, 0, 1000)
    c = oracle_lib.trace(prob, 1000, 2000)
    np.testing.assert_allclose(a["absorbed"], b["absorbed"] + c["absorbed"], rtol=1e-12, atol=1e-22)
    np.testing.assert_allclose(a["images_flat"], b["images_flat"] + c["images_flat"], rtol=1e-12, atol=1e-22)


def test_empty_grid_everything_escapes(oracle_lib):
    grid = W.uniform_grid(4, kr=0.0)
    prob = W.Problem("empty", grid, W.Source(W.SRC_POINT, (0.1, 0.2, 0.3)),
                     W.single_wavelength(), np.array([100], np.uint64),
                     [W.Instrument(10.0, 45.0, 30.0, 2.0, 8)])
    r = oracle_lib.trace(prob, nrec=100)
    assert np.all(r["records"][0, :, 0] == 0)  # no interaction
    np.testing.assert_allclose(r["records"][0, :, 1], 0.01, rtol=1e-15)
    assert r["sed"][0, 0] == pytest.approx(1.0 / (4 * math.pi * 100), rel=1e-14)
    assert np.all(r["absorbed"] == 0)


def test_event_cap_sets_status(oracle_lib):
    prob = W.sphere_problem(50)
    prob.max_events = 1
    r = oracle_lib.trace(prob, nrec=50)
    assert r["status"] & oracle_lib.ERR_EVENT_CAP
    assert np.all(r["records"][0, :, 0] == 1)
    assert np.all(r["records"][0, :, 3] > 0)


def test_zero_packets_is_a_no_op(oracle_lib):
    prob = W.sphere_problem(0)
    r = oracle_lib.trace(prob)
    assert r["status"] == 0 and np.all(r["absorbed"] == 0) and np.all(r["ledger"] == 0)


def test_disk_source_follows_its_distributions(oracle_lib):
    """Launch positions of the exponential-disk source (read from packets on
    a transparent grid, which end where they start): radius ~ Gamma(2, h_R),
    height ~ Laplace(0, h_z), azimuth uniform (Kolmogorov-Smirnov against the
    closed-form distribution functions)."""
    from scipy import stats
    grid = W.uniform_grid(4, half=1000.0, kr=0.0)
    hR, hz = 4.0, 0.4
    prob = W.Problem("disk-launch", grid, W.Source(W.SRC_DISK, (0.0, 0.0, 0.0), h_R=hR, h_z=hz),
                     W.single_wavelength(), np.array([20000], dtype=np.uint64))
    r = oracle_lib.trace(prob, nrec=20000)
    assert r["status"] == 0
    x, y, z = r["records"][0, :, 5], r["records"][0, :, 6], r["records"][0, :, 7]
    R = np.hypot(x, y)
    assert stats.kstest(R, lambda v: 1 - np.exp(-v / hR) * (1 + v / hR)).pvalue > 1e-3
    assert stats.kstest(z, stats.laplace(scale=hz).cdf).pvalue > 1e-3
    phi = np.mod(np.arctan2(y, x), 2 * np.pi) / (2 * np.pi)
    assert stats.kstest(phi, "uniform").pvalue > 1e-3
    assert np.mean(R) == pytest.approx(2 * hR, rel=0.03)


def test_dust_source_cell_frequencies(oracle_lib):
    """The dust-cell source draws cell m with probability emission[m] / sum
    (chi-square over 8 cells of weights 1..8, one dark cell) and a uniform
    point inside it (per-axis fractional positions, Kolmogorov-Smirnov)."""
    from scipy import stats
    from oracle.selfabsorb import cell_cdf
    grid = W.uniform_grid(2, half=1.0, kr=0.0)
    w = np.arange(1.0, 9.0)
    w[5] = 0.0
    cdf, _ = cell_cdf(w[:, None])
    n = 40000
    prob = W.Problem("dust-launch", grid, W.Source(W.SRC_DUST), W.single_wavelength(),
                     np.array([n], dtype=np.uint64))
    r = oracle_lib.trace(prob, nrec=n, cell_cdf=cdf)
    pos = r["records"][0, :, 5:8]
    idx = np.floor(pos + 1.0).astype(int)  # cell size 1 over [-1, 1]
    m = (idx[:, 2] * 2 + idx[:, 1]) * 2 + idx[:, 0]
    counts = np.bincount(m, minlength=8)
    assert counts[5] == 0
    keep = w > 0
    expect = n * w[keep] / w.sum()
    assert stats.chisquare(counts[keep], expect).pvalue > 1e-3
    frac = pos + 1.0 - idx
    for a in range(3):
        assert stats.kstest(frac[:, a], "uniform").pvalue > 1e-3


def test_slab_beam_per_wavelength_extinction_and_luminosity(oracle_lib):
    """Three wavelengths through one pure-absorber slab: wavelength j sees
    optical depth kscale_j tau, launches lsrc_j / npackets_j per packet, so its
    transmitted and per-layer absorbed luminosities are lsrc_j e^{-kscale_j tau}
    and lsrc_j (e^{-kscale_j tau_{l-1}} - e^{-kscale_j tau_l}), exact to rounding."""
    layer_tau = np.array([0.3, 0.9, 0.4], dtype=np.float32).astype(np.float64)
    grid = W.slab_grid(layer_tau)
    kscale = np.array([0.5, 1.0, 2.5])
    lsrc = np.array([1.0, 2.0, 3.0])
    npk = np.array([1, 2, 3], dtype=np.uint64)
    wl = W.Wavelengths(lam=np.array([1.0, 0.55, 0.3]), kscale=kscale, albedo=np.zeros(3), g=np.zeros(3), lsrc=lsrc)
    prob = W.Problem("slab-3", grid, W.Source(W.SRC_BEAM, (0.1, 0.2, 0.0), (0.0, 0.0, 1.0)), wl, npk)
    r = oracle_lib.trace(prob, nrec=3)
    assert r["status"] == 0
    cum = np.concatenate([[0.0], np.cumsum(layer_tau)])
    for j in range(3):
        esc = r["ledger"][j, 2]
        assert esc == pytest.approx(lsrc[j] * math.exp(-kscale[j] * cum[-1]), rel=1e-14)
        got = r["absorbed"][:, j].reshape(grid.nz, -1).sum(axis=1)
        expect = lsrc[j] * (np.exp(-kscale[j] * cum[:-1]) - np.exp(-kscale[j] * cum[1:]))
        np.testing.assert_allclose(got, expect, rtol=1e-13)
        assert r["ledger"][j, 0] == pytest.approx(lsrc[j], rel=1e-15)
