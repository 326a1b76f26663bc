"""Pins of the oracle's octree dust grid: against the regular grid it must
reproduce when every leaf sits on the finest level, against ray marching on
an independent lattice map, against closed forms (slab, chord length), and
against the invariance of the physics under splitting a leaf into eight
children of the same density."""
import dataclasses
import math

import numpy as np
import pytest

from paper_1705_04702_gb300 import workloads as W


def _lattice_map(tree):
    """Leaf index of every finest-lattice cell, painted box by box from the
    leaf list ([z][y][x]); -1 where no leaf lies (a hole)."""
    n = tree.nx
    lat = np.full((n, n, n), -1, dtype=np.int64)
    for m, (lv, ix, iy, iz) in enumerate(tree.leaves.tolist()):
        s = 1 << (tree.max_level - lv)
        lat[iz * s:(iz + 1) * s, iy * s:(iy + 1) * s, ix * s:(ix + 1) * s] = m
    return lat


def _blob_tree(max_level=5, bbox=(-1.0, 1.5, -0.5, 0.5, -2.0, 1.0), delta=2e-3):
    """A tree refined around an off-centre Gaussian blob inside a non-cubic
    root box: leaves of three sizes (levels 3 to 5 with the defaults) meet
    along most rays."""
    def dens(x, y, z):
        return 0.05 + 8.0 * np.exp(-((x - 0.3) ** 2 + (y + 0.1) ** 2 + (z + 0.4) ** 2) / 0.05)
    return W.refine_octree(dens, bbox, max_level, 1, delta)


def _rays(rng, bbox, n):
    lo = np.array(bbox[0::2])
    hi = np.array(bbox[1::2])
    out = []
    for _ in range(n):
        p = lo + rng.random(3) * (hi - lo)
        mu = 2 * rng.random() - 1
        phi = 2 * math.pi * rng.random()
        s = math.sqrt(1 - mu * mu)
        out.append((p, np.array([s * math.cos(phi), s * math.sin(phi), mu])))
    return out


def _exit(bbox, p, k):
    t = math.inf
    for a in range(3):
        if k[a] > 0:
            t = min(t, (bbox[2 * a + 1] - p[a]) / k[a])
        elif k[a] < 0:
            t = min(t, (bbox[2 * a] - p[a]) / k[a])
    return t


def test_generated_trees_tile_their_box(oracle_lib):
    tree = _blob_tree()
    levels = np.bincount(tree.leaves[:, 0], minlength=tree.max_level + 1)
    assert (levels > 0).sum() >= 3 and levels[tree.max_level] > 0
    vol = np.sum(8.0 ** (tree.max_level - tree.leaves[:, 0].astype(np.float64)))
    assert vol == 8.0 ** tree.max_level
    assert np.all(_lattice_map(tree) >= 0)
    assert oracle_lib.octree_valid(tree)


def test_invalid_trees_are_rejected(oracle_lib):
    tree = _blob_tree(max_level=3, delta=2e-2)
    hole = W.Octree(tree.max_level, tree.bbox, tree.leaves[1:], tree.kr[1:])
    dup = W.Octree(tree.max_level, tree.bbox, np.concatenate([tree.leaves, tree.leaves[:1]]),
                   np.concatenate([tree.kr, tree.kr[:1]]))
    parent = tree.leaves[tree.leaves[:, 0] == tree.max_level][:1].copy()
    parent[0, 0] -= 1
    parent[0, 1:] //= 2
    over = W.Octree(tree.max_level, tree.bbox, np.concatenate([tree.leaves, parent]),
                    np.concatenate([tree.kr, tree.kr[:1]]))
    outside = tree.leaves.copy()
    outside[0, 1] = 1 << int(outside[0, 0])
    deep = tree.leaves.copy()
    deep[0, 0] = tree.max_level + 1
    for bad in (hole, dup, over, W.Octree(tree.max_level, tree.bbox, outside, tree.kr),
                W.Octree(tree.max_level, tree.bbox, deep, tree.kr)):
        assert not oracle_lib.octree_valid(bad)
    prob = W.beam_problem(hole, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    assert oracle_lib.trace(prob)["status"] & oracle_lib.ERR_TREE


def test_uniform_tree_paths_equal_the_regular_grid(oracle_lib):
    """Every leaf on the finest level: the same cells and bit-identical
    lengths as the regular grid, for random rays through a clumpy grid."""
    grid = W.torus_grid(16, seed=3)
    tree = W.octree_from_grid(grid)
    pg = W.beam_problem(grid, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    pt = W.beam_problem(tree, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    rng = np.random.default_rng(5)
    for p, k in _rays(rng, grid.bbox, 200):
        c1, l1 = oracle_lib.path(pg, p, k)
        c2, l2 = oracle_lib.path(pt, p, k)
        np.testing.assert_array_equal(c1, c2)
        np.testing.assert_array_equal(l1, l2)


@pytest.mark.parametrize("src", ["point", "dust"])
def test_uniform_tree_trace_equals_the_regular_grid(oracle_lib, src):
    """Whole packet histories, tallies and images bit-identical to the
    regular grid when every leaf sits on the finest level (leaves in the
    grid's cell order), for a point source and for the dust-cell source."""
    from oracle.selfabsorb import cell_cdf
    prob = W.sphere_problem(npackets=1500, n=16)
    prob = dataclasses.replace(prob, instruments=prob.instruments + [W.Instrument(100.0, 70.0, 20.0, 2.0, 32)])
    cdf = None
    if src == "dust":
        rng = np.random.default_rng(2)
        em = rng.random((prob.grid.ncell, 1)) * (prob.grid.kr.ravel()[:, None] > 0)
        cdf, _ = cell_cdf(em)
        prob = dataclasses.replace(prob, source=W.Source(W.SRC_DUST))
    tprob = dataclasses.replace(prob, grid=W.octree_from_grid(prob.grid))
    a = oracle_lib.trace(prob, nrec=1500, cell_cdf=cdf)
    b = oracle_lib.trace(tprob, nrec=1500, cell_cdf=cdf)
    assert a["status"] == 0 and b["status"] == 0
    for key in ("absorbed", "images_flat", "sed", "ledger", "counters", "records"):
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_octree_path_against_fine_marching(oracle_lib):
    """Random rays through a tree with leaves of many sizes inside a
    non-cubic box: the segment lengths sum to the chord to the boundary, and
    every leaf's length agrees with a 2e5-step march that finds leaves on a
    lattice map painted independently from the leaf list."""
    tree = _blob_tree()
    lat = _lattice_map(tree)
    prob = W.beam_problem(tree, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    lo = np.array(tree.bbox[0::2])
    h = (np.array(tree.bbox[1::2]) - lo) / tree.nx
    rng = np.random.default_rng(11)
    nstep = 200_000
    for p, k in _rays(rng, tree.bbox, 40):
        cells, lens = oracle_lib.path(prob, p, k)
        texit = _exit(tree.bbox, p, k)
        assert lens.sum() == pytest.approx(texit, rel=1e-12)
        assert np.all(lens > 0)
        assert np.all(cells[1:] != cells[:-1])
        assert len(np.unique(cells)) == len(cells)  # a box is entered once
        dt = texit / nstep
        t = (np.arange(nstep) + 0.5) * dt
        pts = p[None, :] + t[:, None] * k[None, :]
        j = np.clip(np.floor((pts - lo) / h).astype(np.int64), 0, tree.nx - 1)
        leaf = lat[j[:, 2], j[:, 1], j[:, 0]]
        march = np.bincount(leaf, minlength=tree.ncell) * dt
        seg = np.zeros(tree.ncell)
        np.add.at(seg, cells, lens)
        assert np.max(np.abs(march - seg)) <= 1.01 * dt
        long_ = cells[lens > 2 * dt]
        order = leaf[np.r_[True, leaf[1:] != leaf[:-1]]]
        order = order[np.isin(order, long_)]
        np.testing.assert_array_equal(order, long_)


def test_octree_slab_beam_pure_absorber(oracle_lib):
    """Layered pure absorber on a tree whose leaves along the beam come in
    three sizes: transmission e^{-tau/mu} and the absorption of every layer
    e^{-tau_{l-1}/mu} - e^{-tau_l/mu}, exact to rounding."""
    layer_tau = np.array([0.2, 0.7, 0.5, 1.6], dtype=np.float32).astype(np.float64)
    base = W.Grid(4, 4, 4, (-8.0, 8.0, -8.0, 8.0, 0.0, 4.0),
                  np.repeat(layer_tau.astype(np.float32), 16).reshape(4, 4, 4))
    tree = dataclasses.replace(W.octree_from_grid(base), max_level=4)
    col = np.nonzero((tree.leaves[:, 1] == 1) & (tree.leaves[:, 2] == 2) & (tree.leaves[:, 3] >= 1))[0]
    tree = W.split_leaves(tree, col)
    tree = W.split_leaves(tree, np.nonzero(tree.leaves[:, 0] == 3)[0][::3])
    assert np.array_equal(np.unique(tree.leaves[:, 0]), [2, 3, 4])
    assert oracle_lib.octree_valid(tree)
    lo_z, hi_z = tree.boxes()[0][:, 2], tree.boxes()[1][:, 2]
    layer = np.floor(lo_z).astype(int)
    assert np.all(hi_z <= layer + 1)
    for mu in (1.0, 0.6):
        k = (math.sqrt(1 - mu * mu), 0.0, mu)
        prob = W.beam_problem(tree, (-0.3, 0.2, 0.0), k, npackets=1, albedo=0.0)
        r = oracle_lib.trace(prob, nrec=1)
        assert r["status"] == 0
        rec = r["records"][0, 0]
        assert rec[1] == pytest.approx(math.exp(-layer_tau.sum() / mu), rel=1e-14)
        cum = np.concatenate([[0.0], np.cumsum(layer_tau)]) / mu
        expect = np.exp(-cum[:-1]) - np.exp(-cum[1:])
        got = np.bincount(layer, weights=r["absorbed"][:, 0], minlength=4)
        np.testing.assert_allclose(got, expect, rtol=1e-13)


def test_split_leaves_leave_the_physics_unchanged(oracle_lib):
    """Splitting leaves into eight children of the same density changes only
    where the paths are cut: the packet histories agree to rounding and every
    parent's absorption equals the sum over its children."""
    tree = W.refine_octree(W.disk_density(), (-24.0, 24.0, -24.0, 24.0, -24.0, 24.0), 7, 3, 2e-3)
    rng = np.random.default_rng(4)
    cand = np.nonzero(tree.leaves[:, 0] < tree.max_level)[0]
    which = np.sort(rng.choice(cand, size=min(400, cand.size), replace=False))
    split = W.split_leaves(tree, which)
    a = oracle_lib.trace(W.octree_problem(tree, 3000, npx=64), nrec=3000)
    b = oracle_lib.trace(W.octree_problem(split, 3000, npx=64), nrec=3000)
    ra, rb = a["records"][0], b["records"][0]
    same = ra[:, 0] == rb[:, 0]
    assert same.mean() >= 0.999
    rel = np.abs(ra[same] - rb[same]) / np.maximum(np.abs(ra[same]), 1e-300)
    big = np.abs(ra[same]) > 1e-12 * np.abs(ra[same]).max(axis=0)
    assert np.max(rel[big]) < 1e-9
    nk = tree.ncell - which.size
    keep = np.setdiff1d(np.arange(tree.ncell), which)
    tot = a["absorbed"].sum()
    np.testing.assert_allclose(b["absorbed"][:nk, 0], a["absorbed"][keep, 0], rtol=0, atol=1e-9 * tot)
    children = b["absorbed"][nk:, 0].reshape(-1, 8).sum(axis=1)
    np.testing.assert_allclose(children, a["absorbed"][which, 0], rtol=0, atol=1e-9 * tot)


def test_octree_energy_closes(oracle_lib):
    tree = _blob_tree()
    prob = W.Problem("blob", tree, W.Source(W.SRC_POINT, (0.3, -0.1, -0.4)),
                     W.powerlaw_wavelengths(3, 0.2, 2.0), np.array([800, 500, 300], dtype=np.uint64),
                     [W.Instrument(50.0, 30.0, 10.0, 3.0, 16)])
    r = oracle_lib.trace(prob)
    assert r["status"] == 0
    led = r["ledger"]
    np.testing.assert_allclose(led[:, 0], led[:, 1] + led[:, 2] + led[:, 3], rtol=1e-12)
    np.testing.assert_allclose(r["absorbed"].sum(axis=0), led[:, 1], rtol=1e-12)


def test_octree_dust_source_stays_in_its_leaf(oracle_lib):
    """Transparent tree, all emission in one small leaf: every packet leaves
    from inside that leaf's box (a packet with nothing on its path ends where
    it started)."""
    from oracle.selfabsorb import cell_cdf
    tree = _blob_tree()
    tree = dataclasses.replace(tree, kr=np.zeros_like(tree.kr))
    m = int(np.nonzero(tree.leaves[:, 0] == tree.max_level)[0][7])
    em = np.zeros((tree.ncell, 1))
    em[m] = 1.0
    cdf, _ = cell_cdf(em)
    prob = W.Problem("dust", tree, W.Source(W.SRC_DUST), W.single_wavelength(), np.array([500], dtype=np.uint64))
    r = oracle_lib.trace(prob, nrec=500, cell_cdf=cdf)
    a, b = tree.boxes()
    x = r["records"][0, :, 5:8]
    assert np.all(x >= a[m]) and np.all(x <= b[m])
    assert np.ptp(x, axis=0).min() > 0.5 * (b[m] - a[m]).min()


def test_refinement_follows_the_mass_criterion():
    """The input generator's rule, as stated for the workloads: every box is
    split down to min_level; beyond it a leaf below max_level holds at most
    delta of the total mass, the parent of every deeper leaf held more, and
    the leaves come in strictly increasing Morton order."""
    bbox = (-24.0, 24.0, -24.0, 24.0, -24.0, 24.0)
    dens = W.disk_density()
    max_level, min_level, delta, sub = 7, 3, 2e-4, 2
    tree = W.refine_octree(dens, bbox, max_level, min_level, delta, sub=sub)
    lo = np.array(bbox[0::2])
    ext = np.array(bbox[1::2]) - lo
    off = (np.arange(sub) + 0.5) / sub

    def mass(level, cell):
        h = ext / 2 ** level
        pts = np.array([lo + (np.asarray(cell) + np.array([a, b, c])) * h for a in off for b in off for c in off])
        return dens(pts[:, 0], pts[:, 1], pts[:, 2]).mean() * np.prod(h)

    n = 2 ** min_level
    total = sum(mass(min_level, (i, j, k)) for i in range(n) for j in range(n) for k in range(n))
    rng = np.random.default_rng(0)
    lv = tree.leaves[:, 0]
    assert lv.min() >= min_level and lv.max() <= max_level
    for m in rng.choice(tree.ncell, size=300, replace=False):
        level, ix, iy, iz = (int(v) for v in tree.leaves[m])
        if level < max_level:
            assert mass(level, (ix, iy, iz)) <= delta * total * (1 + 1e-12)
        if level > min_level:
            assert mass(level - 1, (ix // 2, iy // 2, iz // 2)) > delta * total * (1 - 1e-12)
    corner = tree.leaves[:, 1:].astype(np.int64) << (max_level - lv[:, None].astype(np.int64))
    key = np.zeros(tree.ncell, dtype=np.int64)
    for bit in range(max_level):
        for a in range(3):
            key |= ((corner[:, a] >> bit) & 1) << (3 * bit + a)
    assert np.all(np.diff(key) > 0)
    c = tree.centres()
    np.testing.assert_array_equal(tree.kr, dens(c[:, 0], c[:, 1], c[:, 2]).astype(np.float32))


def test_octree_descriptions_refuse_bad_inputs():
    """Host-side checks of the octree description helpers: a uniform tree
    needs a 2^L cube, and a finest-level leaf cannot be split."""
    with pytest.raises(ValueError):
        W.octree_from_grid(W.uniform_grid(6))
    with pytest.raises(ValueError):
        W.octree_from_grid(W.Grid(4, 4, 8, (-1, 1, -1, 1, -1, 1), np.zeros((8, 4, 4), np.float32)))
    tree = W.octree_from_grid(W.uniform_grid(4))
    with pytest.raises(ValueError):
        W.split_leaves(tree, [0])
    deeper = dataclasses.replace(tree, max_level=3)
    split = W.split_leaves(deeper, [0, 5])
    assert split.ncell == tree.ncell + 14
    a, b = split.boxes()
    np.testing.assert_allclose(np.prod(b - a, axis=1).sum(), 8.0, rtol=1e-14)
