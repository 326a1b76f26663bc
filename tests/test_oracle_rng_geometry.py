"""Pins of the oracle's building blocks against values fixed outside it:
published Philox known answers, exact geometry, the Henyey-Greenstein CDF,
and the invariants of the direction rotation."""
import math
import os

import numpy as np
import pytest

from paper_1705_04702_gb300 import workloads as W


def _philox_kat():
    """Known-answer vectors of Philox4x32-10 from tests/golden (cited there):
    (counter, key) -> output."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    out = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        ctr, key, res = (tuple(int(w, 16) for w in part.split()) for part in line.split("|"))
        out.append((ctr, key, res))
    return out


PHILOX_KAT = _philox_kat()


@pytest.mark.parametrize("ctr,key,expect", PHILOX_KAT)
def test_philox_known_answers(oracle_lib, ctr, key, expect):
    assert len(PHILOX_KAT) == 3
    assert tuple(oracle_lib.philox4x32_10(ctr, key)) == expect


def test_uniform_is_exact_in_fp32(oracle_lib):
    # u = (k + 1/2) 2^-23 for the top 23 bits k: endpoints and FP32 exactness
    assert oracle_lib.uniform(0) == 2.0 ** -24
    assert oracle_lib.uniform(0xffffffff) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(3)
    for x in rng.integers(0, 2 ** 32, 2000, dtype=np.uint64):
        u = oracle_lib.uniform(int(x))
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
        assert u == ((int(x) >> 9) * 2 + 1) / 2 ** 24


# ---------------------------------------------------------------------------
# geometry: the oracle's ray / grid intersection
# ---------------------------------------------------------------------------
def _prob(grid):
    return W.beam_problem(grid, (0, 0, 0), (0, 0, 1))


def test_path_26_neighbour_directions(oracle_lib):
    """From the centre of the middle cell of a 3^3 unit-cell grid, every
    direction (a,b,c) in {-1,0,1}^3 runs half a cell through the middle cell,
    then crosses exactly into the face/edge/corner neighbour (a,b,c) for a
    full cell (in units of |(a,b,c)|), including the edge and corner ties."""
    grid = W.uniform_grid(3, half=1.5)
    prob = _prob(grid)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            for c in (-1, 0, 1):
                if a == b == c == 0:
                    continue
                nrm = math.sqrt(a * a + b * b + c * c)
                k = (a / nrm, b / nrm, c / nrm)
                cells, lens = oracle_lib.path(prob, (0.0, 0.0, 0.0), k)
                assert len(cells) == 2, (a, b, c, cells, lens)
                assert cells[0] == 13
                assert cells[1] == ((1 + c) * 3 + (1 + b)) * 3 + (1 + a)
                # half a cell in the middle cell, a full cell in the neighbour,
                # both measured along the ray
                assert lens[0] == pytest.approx(0.5 * nrm, rel=1e-14)
                assert lens[1] == pytest.approx(nrm, rel=1e-14)


def _brute_march(grid, p, k, nstep=200_000):
    """Fine ray-marching: cell of every sample point along the ray up to the
    exit, counted with a fixed step -> per-cell length with error <= 2 steps."""
    x0, x1, y0, y1, z0, z1 = grid.bbox
    lo = np.array([x0, y0, z0])
    hi = np.array([x1, y1, z1])
    n = np.array([grid.nx, grid.ny, grid.nz])
    with np.errstate(divide="ignore"):
        tb = np.where(np.asarray(k) > 0, (hi - p) / k, np.where(np.asarray(k) < 0, (lo - p) / k, np.inf))
    texit = tb.min()
    h = texit / nstep
    t = (np.arange(nstep) + 0.5) * h
    pts = p[None, :] + t[:, None] * np.asarray(k)[None, :]
    idx = np.clip(np.floor((pts - lo) / ((hi - lo) / n)).astype(np.int64), 0, n - 1)
    m = (idx[:, 2] * grid.ny + idx[:, 1]) * grid.nx + idx[:, 0]
    lengths = np.bincount(m, minlength=grid.ncell) * h
    return texit, lengths, h


def test_path_matches_brute_force_marching(oracle_lib):
    rng = np.random.default_rng(11)
    for trial in range(12):
        nx, ny, nz = rng.integers(1, 9, 3)
        grid = W.Grid(int(nx), int(ny), int(nz), (-1.3, 0.7, -0.4, 2.0, -1.0, 1.0),
                      np.ones((nz, ny, nx), np.float32))
        prob = _prob(grid)
        lo = np.array([-1.3, -0.4, -1.0])
        hi = np.array([0.7, 2.0, 1.0])
        p = lo + rng.random(3) * (hi - lo)
        k = rng.normal(size=3)
        if trial % 4 == 0:
            k[trial % 3] = 0.0  # a direction component exactly zero
        k /= np.linalg.norm(k)
        cells, lens = oracle_lib.path(prob, p, k)
        texit, ref, h = _brute_march(grid, p, k)
        # sum of segment lengths equals the chord to the exit
        assert lens.sum() == pytest.approx(texit, rel=1e-12)
        got = np.zeros(grid.ncell)
        np.add.at(got, cells, lens)
        assert np.max(np.abs(got - ref)) <= 2.5 * h
        # consecutive cells are grid neighbours
        ix, iy, iz = cells % grid.nx, (cells // grid.nx) % grid.ny, cells // (grid.nx * grid.ny)
        steps = np.abs(np.diff(ix)) + np.abs(np.diff(iy)) + np.abs(np.diff(iz))
        assert np.all((steps >= 1) & (np.maximum.reduce([np.abs(np.diff(ix)), np.abs(np.diff(iy)),
                                                          np.abs(np.diff(iz))]) == 1))


def test_path_from_boundary_outward_is_empty(oracle_lib):
    grid = W.uniform_grid(4)
    cells, lens = oracle_lib.path(_prob(grid), (1.0, 0.2, 0.1), (1.0, 0.0, 0.0))
    assert len(cells) == 0


# ---------------------------------------------------------------------------
# Henyey-Greenstein sampling and direction rotation
# ---------------------------------------------------------------------------
def _hg_cdf(g, mu):
    # analytic cumulative distribution of mu under HG, P(mu' <= mu)
    return (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))


@pytest.mark.parametrize("g", [0.6, -0.3, 0.9, 0.05])
def test_hg_sampler_inverts_the_cdf(oracle_lib, g):
    u = (np.arange(20000) + 0.5) / 20000
    mu = np.array([oracle_lib.hg_mu(g, x) for x in u])
    assert np.all(np.diff(mu) > 0)
    np.testing.assert_allclose(_hg_cdf(g, mu), u, rtol=0, atol=2e-12)
    # mean cosine of HG equals g
    assert mu.mean() == pytest.approx(g, abs=2e-4)


def test_hg_isotropic_limit(oracle_lib):
    for u in (1e-3, 0.25, 0.5, 0.8):
        assert oracle_lib.hg_mu(0.0, u) == 2 * u - 1
        assert oracle_lib.hg_mu(1e-9, u) == 2 * u - 1


def test_rotation_invariants(oracle_lib):
    rng = np.random.default_rng(5)
    ks = [np.array([0.0, 0.0, 1.0]), np.array([0.0, 0.0, -1.0])]
    for _ in range(40):
        k = rng.normal(size=3)
        ks.append(k / np.linalg.norm(k))
    for k in ks:
        for mu in (-0.9, -0.2, 0.0, 0.3, 0.97):
            phi = rng.random() * 2 * math.pi
            a = oracle_lib.rotate(k, mu, phi)
            b = oracle_lib.rotate(k, mu, phi + math.pi)
            assert np.linalg.norm(a) == pytest.approx(1.0, abs=1e-12)
            assert float(a @ k) == pytest.approx(mu, abs=1e-12)
            # azimuths phi and phi+pi are mirror images about k
            np.testing.assert_allclose(a + b, 2 * mu * k, atol=1e-12)
