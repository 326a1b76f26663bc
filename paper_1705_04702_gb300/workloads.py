"""Seeded synthetic inputs for the photon-packet life cycle.

This module only *describes* problems: dust-grid densities from analytic
geometries, wavelength tables, packet counts, instruments.  It contains none
of the radiative-transfer arithmetic, so the CUDA library and the CPU oracle
can both consume its output without sharing any of the method's code.

The paper's own test model (a spiral galaxy with bulge, ring and arms on a
256,000-cell Cartesian grid, Sect. 7.2) and its ERIS run (Sect. 7.9) are not
available as data; the generators below stand in for them with the same
structure (exponential disks, a clumpy torus) and the grid, wavelength and
packet counts listed in the workload descriptions.

Conventions
-----------
* Grid: ``kr`` has shape ``(nz, ny, nx)`` (x fastest), dtype float32; it is
  the extinction coefficient kappa*rho [1/length] at the reference wavelength
  (0.55 micron).  The values are rounded to float32 once, so the FP64 and the
  FP32 form of the tracer see exactly the same numbers.
* Wavelength table: ``kscale`` = kappa_ext(lambda)/kappa_ext(ref),
  ``albedo``, ``g`` (Henyey-Greenstein asymmetry), ``lsrc`` (luminosity the
  source emits in that wavelength bin), ``npk`` (packets launched).
* Instruments: distant observers (distance, inclination, azimuth in degrees,
  square field of view ``fov`` centred on the origin, ``npx`` x ``npx``).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

SRC_POINT, SRC_DISK, SRC_BEAM, SRC_DUST = 0, 1, 2, 3


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    bbox: tuple  # (xmin, xmax, ymin, ymax, zmin, zmax)
    kr: np.ndarray  # float32 (nz, ny, nx)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny * self.nz

    def centres(self):
        """Cell-centre coordinates as three 1-D arrays (x, y, z)."""
        x0, x1, y0, y1, z0, z1 = self.bbox
        xs = x0 + (np.arange(self.nx) + 0.5) * (x1 - x0) / self.nx
        ys = y0 + (np.arange(self.ny) + 0.5) * (y1 - y0) / self.ny
        zs = z0 + (np.arange(self.nz) + 0.5) * (z1 - z0) / self.nz
        return xs, ys, zs


@dataclass
class Octree:
    """Adaptive octree dust grid (the grid kind of the paper's ERIS run,
    Sect. 7.9, with up to 13 division levels).  The root box ``bbox`` is split
    into 8 equal boxes, recursively; leaf m has level ``leaves[m, 0]`` and
    integer position ``leaves[m, 1:4]`` (x, y, z) among the 2^level boxes of
    that level along each axis, so it spans lattice cells
    [i << (L - level), (i + 1) << (L - level)) of the finest lattice
    (L = ``max_level``, 2^L cells per axis).  ``kr`` [nleaf] float32 is the
    extinction coefficient as for the regular grid; the leaves are the cells
    (absorbed tables, emission and dust-source tables are indexed by leaf)."""
    max_level: int
    bbox: tuple
    leaves: np.ndarray  # int32 (nleaf, 4): level, ix, iy, iz
    kr: np.ndarray  # float32 (nleaf,)

    @property
    def nx(self) -> int:
        return 1 << self.max_level

    ny = nx
    nz = nx

    @property
    def ncell(self) -> int:
        return int(self.leaves.shape[0])

    def boxes(self):
        """Lower and upper corners of every leaf, (nleaf, 3) each."""
        lo = np.array(self.bbox[0::2], dtype=np.float64)
        ext = np.array(self.bbox[1::2], dtype=np.float64) - lo
        h = ext[None, :] / (2.0 ** self.leaves[:, :1].astype(np.float64))
        a = lo[None, :] + self.leaves[:, 1:].astype(np.float64) * h
        return a, a + h

    def centres(self):
        a, b = self.boxes()
        return 0.5 * (a + b)


@dataclass
class Source:
    kind: int = SRC_POINT
    pos: tuple = (0.0, 0.0, 0.0)
    dir: tuple = (0.0, 0.0, 1.0)
    h_R: float = 0.0
    h_z: float = 0.0


@dataclass
class Wavelengths:
    lam: np.ndarray
    kscale: np.ndarray
    albedo: np.ndarray
    g: np.ndarray
    lsrc: np.ndarray

    @property
    def n(self) -> int:
        return int(self.lam.shape[0])


@dataclass
class Instrument:
    distance: float
    inclination: float  # degrees
    azimuth: float  # degrees
    fov: float
    npx: int


@dataclass
class Problem:
    name: str
    grid: Grid
    source: Source
    wl: Wavelengths
    npk: np.ndarray  # uint64 per wavelength
    instruments: list = field(default_factory=list)
    seed: int = 1
    w_min: float = 1e-4
    max_events: int = 10000
    phase: int = 0

    @property
    def total_packets(self) -> int:
        return int(np.sum(self.npk, dtype=np.uint64))

    def with_packets(self, npk) -> "Problem":
        npk = np.broadcast_to(np.asarray(npk, dtype=np.uint64), (self.wl.n,)).copy()
        return dataclasses.replace(self, npk=npk)


# ----------------------------------------------------------------------------
# wavelength tables
# ----------------------------------------------------------------------------
def single_wavelength(albedo=0.5, g=0.6, lam=0.55, lsrc=1.0) -> Wavelengths:
    return Wavelengths(lam=np.array([lam]), kscale=np.array([1.0]),
                       albedo=np.array([albedo], dtype=np.float64),
                       g=np.array([g], dtype=np.float64),
                       lsrc=np.array([lsrc], dtype=np.float64))


def powerlaw_wavelengths(n, lam_min, lam_max, slope=-1.2, alb_short=0.7,
                         alb_long=0.3, g=0.6, lam_ref=0.55) -> Wavelengths:
    """``n`` log-spaced wavelengths [micron]; kappa ~ lambda^slope relative to
    the reference wavelength; albedo linear in log(lambda) from ``alb_short``
    at the shortest to ``alb_long`` at the longest wavelength; flat source
    spectrum (unit luminosity per bin)."""
    lam = np.geomspace(lam_min, lam_max, n)
    kscale = (lam / lam_ref) ** slope
    frac = (np.log(lam) - np.log(lam_min)) / max(np.log(lam_max) - np.log(lam_min), 1e-300)
    albedo = alb_short + (alb_long - alb_short) * frac
    return Wavelengths(lam=lam, kscale=kscale, albedo=albedo,
                       g=np.full(n, g), lsrc=np.ones(n))


# ----------------------------------------------------------------------------
# dust grids
# ----------------------------------------------------------------------------
def uniform_grid(n, half=1.0, kr=1.0, nxyz=None) -> Grid:
    nx, ny, nz = nxyz if nxyz is not None else (n, n, n)
    arr = np.full((nz, ny, nx), kr, dtype=np.float32)
    return Grid(nx, ny, nz, (-half, half, -half, half, -half, half), arr)


def sphere_grid(n=32, radius=1.0, kr_in=1.0, sub=8) -> Grid:
    """Uniform sphere of extinction coefficient ``kr_in`` inside ``radius``
    on an ``n``^3 grid over [-1,1]^3; each cell carries kr_in times the
    fraction of ``sub``^3 sub-sample points that fall inside the sphere."""
    h = 2.0 / n
    off = (np.arange(sub) + 0.5) / sub
    c = -1.0 + (np.arange(n)[:, None] + off[None, :]) * h  # (n, sub)
    c2 = (c * c)  # squared coordinate of every sub-sample
    # inside[i,a, j,b, k,c] via broadcasting on squared coordinates
    zz = c2[:, :, None, None, None, None]
    yy = c2[None, None, :, :, None, None]
    xx = c2[None, None, None, None, :, :]
    inside = (xx + yy + zz) <= radius * radius
    frac = inside.mean(axis=(1, 3, 5))  # (nz, ny, nx)
    return Grid(n, n, n, (-1.0, 1.0, -1.0, 1.0, -1.0, 1.0),
                (kr_in * frac).astype(np.float32))


def disk_grid(n=256, h_R=6.0, h_z=0.25, tau_face=1.0, xy_half=24.0, z_half=3.0,
              nxyz=None) -> Grid:
    """Exponential dust disk kr = kr0 exp(-R/h_R - |z|/h_z), evaluated at the
    cell centres, with kr0 = tau_face / (2 h_z) so that the face-on optical
    depth through the centre is ``tau_face``."""
    nx, ny, nz = nxyz if nxyz is not None else (n, n, n)
    g = Grid(nx, ny, nz, (-xy_half, xy_half, -xy_half, xy_half, -z_half, z_half),
             np.zeros((nz, ny, nx), dtype=np.float32))
    xs, ys, zs = g.centres()
    kr0 = tau_face / (2.0 * h_z)
    R = np.sqrt(xs[None, :] ** 2 + ys[:, None] ** 2)  # (ny, nx)
    g.kr = (kr0 * np.exp(-R[None, :, :] / h_R - np.abs(zs)[:, None, None] / h_z)).astype(np.float32)
    return g


def torus_grid(n=256, seed=1, r_in=0.05, r_out=1.0, half_opening_deg=50.0,
               p=1.0, q=6.0, tau_eq=10.0, clump_fraction=0.05, clump_contrast=100.0) -> Grid:
    """Clumpy two-phase dust torus on [-1,1]^3: smooth density
    kr0 r^-p exp(-q |cos theta|) for r_in <= r <= r_out within
    ``half_opening_deg`` of the equatorial plane, normalised so that the smooth
    equatorial optical depth from r_in to r_out is ``tau_eq``; each dusty cell
    independently (numpy generator seeded with ``seed``) becomes a clump of
    ``clump_contrast`` times the smooth density with probability
    ``clump_fraction``."""
    g = Grid(n, n, n, (-1.0, 1.0, -1.0, 1.0, -1.0, 1.0),
             np.zeros((n, n, n), dtype=np.float32))
    xs, ys, zs = g.centres()
    X = xs[None, None, :]
    Y = ys[None, :, None]
    Z = zs[:, None, None]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    cos_t = np.abs(Z) / np.maximum(r, 1e-300)
    if p == 1.0:
        norm = np.log(r_out / r_in)
    else:
        norm = (r_out ** (1 - p) - r_in ** (1 - p)) / (1 - p)
    kr0 = tau_eq / norm
    inside = (r >= r_in) & (r <= r_out) & (cos_t <= np.sin(np.radians(half_opening_deg)))
    dens = np.where(inside, kr0 * np.maximum(r, r_in) ** (-p) * np.exp(-q * cos_t), 0.0)
    rng = np.random.default_rng(seed)
    clump = rng.random(dens.shape) < clump_fraction
    dens = np.where(clump & inside, dens * clump_contrast, dens)
    g.kr = dens.astype(np.float32)
    return g


def slab_grid(taus_per_layer, nxy=4, half_xy=1000.0, z0=0.0, dz=1.0) -> Grid:
    """Plane-parallel slab: layer l (along z) has optical depth per unit
    length ``taus_per_layer[l] / dz``; wide in x and y so that oblique beams
    stay inside."""
    t = np.asarray(taus_per_layer, dtype=np.float64)
    nz = t.shape[0]
    arr = np.empty((nz, nxy, nxy), dtype=np.float32)
    arr[:] = (t / dz).astype(np.float32)[:, None, None]
    return Grid(nxy, nxy, nz, (-half_xy, half_xy, -half_xy, half_xy, z0, z0 + nz * dz), arr)


# ----------------------------------------------------------------------------
# octree dust grids
# ----------------------------------------------------------------------------
_OCTANTS = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.int64)


def morton_order(leaves, max_level):
    """Permutation that sorts leaves by the Morton (Z-order) key of their
    lower corner on the finest lattice."""
    corner = leaves[:, 1:].astype(np.int64) << (max_level - leaves[:, :1].astype(np.int64))
    key = np.zeros(leaves.shape[0], dtype=np.int64)
    for bit in range(max_level):
        for a in range(3):
            key |= ((corner[:, a] >> bit) & 1) << (3 * bit + a)
    return np.argsort(key, kind="stable")


def octree_from_grid(grid: Grid) -> Octree:
    """The uniform octree of a regular 2^L x 2^L x 2^L grid: every cell is a
    leaf of level L, in the grid's cell order."""
    n = grid.nx
    L = n.bit_length() - 1
    if not (grid.nx == grid.ny == grid.nz and n == 1 << L and L >= 1):
        raise ValueError("the grid must be 2^L cells along every axis")
    iz, iy, ix = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    leaves = np.stack([np.full(ix.size, L), ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.int32)
    return Octree(L, tuple(grid.bbox), leaves, np.ascontiguousarray(grid.kr, dtype=np.float32).ravel())


def refine_octree(density, bbox, max_level, min_level, delta, sub=2) -> Octree:
    """Octree from a density function by the dust-mass criterion: every box
    is split down to ``min_level``; beyond it a box is split while its dust
    mass exceeds ``delta`` times the total and its level is below
    ``max_level``.  A box's mass is its volume times the mean of ``density``
    at ``sub``^3 regularly spaced interior points; the total is the sum over
    the ``min_level`` boxes.  Leaves carry ``density`` at their centre (as the
    regular grids do) and come in Morton order."""
    lo = np.array(bbox[0::2], dtype=np.float64)
    ext = np.array(bbox[1::2], dtype=np.float64) - lo
    off = (np.arange(sub) + 0.5) / sub
    o = np.stack([v.ravel() for v in np.meshgrid(off, off, off, indexing="ij")], axis=1)

    def mass(cells, level):
        h = ext / (1 << level)
        out = np.empty(len(cells))
        for a in range(0, len(cells), 1 << 20):
            c = cells[a:a + (1 << 20)].astype(np.float64)
            pts = lo + (c[:, None, :] + o[None]) * h
            out[a:a + len(c)] = density(pts[..., 0], pts[..., 1], pts[..., 2]).mean(axis=1) * np.prod(h)
        return out

    n = 1 << min_level
    base = np.stack([v.ravel() for v in np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")],
                    axis=1).astype(np.int64)
    total = mass(base, min_level).sum()
    cells = np.zeros((1, 3), dtype=np.int64)
    out = []
    for level in range(max_level + 1):
        if level < min_level:
            split = np.ones(len(cells), dtype=bool)
        else:
            split = (mass(cells, level) > delta * total) & (level < max_level)
        keep = cells[~split]
        if len(keep):
            out.append(np.concatenate([np.full((len(keep), 1), level, dtype=np.int64), keep], axis=1))
        parents = cells[split]
        if not len(parents):
            break
        cells = (2 * parents[:, None, :] + _OCTANTS[None]).reshape(-1, 3)
    leaves = np.concatenate(out).astype(np.int32)
    leaves = leaves[morton_order(leaves, max_level)]
    t = Octree(max_level, tuple(float(v) for v in bbox), leaves, np.zeros(len(leaves), dtype=np.float32))
    c = t.centres()
    t.kr = density(c[:, 0], c[:, 1], c[:, 2]).astype(np.float32)
    return t


def split_leaves(tree: Octree, which) -> Octree:
    """The same dust distribution with the leaves ``which`` each split into
    their 8 children (same extinction coefficient); the children follow the
    untouched leaves, in octant order."""
    which = np.unique(np.asarray(which, dtype=np.int64))
    lf = tree.leaves[which].astype(np.int64)
    if np.any(lf[:, 0] >= tree.max_level):
        raise ValueError("cannot split a leaf of the finest level")
    ch = np.concatenate([np.repeat(lf[:, :1] + 1, 8, axis=0),
                         (2 * lf[:, None, 1:] + _OCTANTS[None]).reshape(-1, 3)], axis=1).astype(np.int32)
    keep = np.setdiff1d(np.arange(tree.ncell), which)
    return Octree(tree.max_level, tree.bbox, np.concatenate([tree.leaves[keep], ch]),
                  np.concatenate([tree.kr[keep], np.repeat(tree.kr[which], 8)]).astype(np.float32))


def disk_density(h_R=6.0, h_z=0.25, tau_face=1.0):
    """The exponential dust disk of ``disk_grid`` as a function of position."""
    kr0 = tau_face / (2.0 * h_z)

    def f(x, y, z):
        return kr0 * np.exp(-np.sqrt(x * x + y * y) / h_R - np.abs(z) / h_z)
    return f


def disk_octree(max_level=13, delta=1.35e-6, min_level=4, half=24.0) -> Octree:
    """The exponential dust disk on an octree over the cube [-half, half]^3,
    refined by dust mass: with the defaults about 8.2 million leaves (the
    size of the paper's ERIS grid) down to level 11, capped at 13 levels."""
    return refine_octree(disk_density(), (-half, half, -half, half, -half, half), max_level, min_level, delta)


def octree_problem(tree: Octree, npackets=1_000_000, nlambda=1, npx=512, seed=1, albedo=0.5, g=0.6) -> Problem:
    """The exponential-disk galaxy (stellar disk h_R=4, h_z=0.4; three
    instruments at 0/60/90 degrees) on an octree dust grid; wavelengths as in
    ``disk_problem``."""
    wl = single_wavelength(albedo=albedo, g=g) if nlambda == 1 else powerlaw_wavelengths(nlambda, 0.1, 5.0, g=g)
    fov = float(tree.bbox[1] - tree.bbox[0])
    return Problem(
        name=f"octree{tree.ncell}_l{nlambda}",
        grid=tree,
        source=Source(SRC_DISK, (0.0, 0.0, 0.0), h_R=4.0, h_z=0.4),
        wl=wl,
        npk=np.full(wl.n, npackets, dtype=np.uint64),
        instruments=galaxy_instruments(npx, fov=fov),
        seed=seed,
    )


# ----------------------------------------------------------------------------
# the five workloads (sphere, disk FP64-vs-FP32, disk 40 lambda, torus 200
# lambda, learned emission) and scaled-down variants for tests
# ----------------------------------------------------------------------------
def sphere_problem(npackets=100_000, n=32, albedo=0.5, g=0.6, seed=1) -> Problem:
    """Point source (L=1) at the centre of a uniform dust sphere of radius 1
    and radial optical depth 1, 32^3 grid, one wavelength, one face-on
    instrument at distance 100 with 64x64 pixels."""
    return Problem(
        name=f"sphere{n}",
        grid=sphere_grid(n),
        source=Source(SRC_POINT, (0.0, 0.0, 0.0)),
        wl=single_wavelength(albedo=albedo, g=g),
        npk=np.array([npackets], dtype=np.uint64),
        instruments=[Instrument(100.0, 0.0, 0.0, 2.0, 64)],
        seed=seed,
    )


def galaxy_instruments(npx=512, fov=48.0, distance=100.0):
    return [Instrument(distance, inc, 0.0, fov, npx) for inc in (0.0, 60.0, 90.0)]


def disk_problem(npackets=100_000_000, n=256, nlambda=1, npx=512, seed=1,
                 albedo=0.5, g=0.6) -> Problem:
    """Exponential-disk galaxy: stellar disk h_R=4, h_z=0.4; dust disk
    h_R=6, h_z=0.25, face-on tau_V=1; 3 instruments at inclinations 0/60/90
    degrees.  ``nlambda == 1``: one optical wavelength, ``npackets`` packets.
    ``nlambda > 1``: log-spaced 0.1-5 micron with kappa ~ lambda^-1.2 and
    albedo 0.7 -> 0.3, ``npackets`` packets per wavelength."""
    grid = disk_grid(n)
    if nlambda == 1:
        wl = single_wavelength(albedo=albedo, g=g)
    else:
        wl = powerlaw_wavelengths(nlambda, 0.1, 5.0, g=g)
    return Problem(
        name=f"disk{n}_l{nlambda}",
        grid=grid,
        source=Source(SRC_DISK, (0.0, 0.0, 0.0), h_R=4.0, h_z=0.4),
        wl=wl,
        npk=np.full(wl.n, npackets, dtype=np.uint64),
        instruments=galaxy_instruments(npx, fov=48.0),
        seed=seed,
    )


def uneven_packet_counts(nlambda, lo=1e5, hi=2e7, seed=1, scale=1.0):
    """Packet counts drawn log-uniform in [lo, hi] with numpy's generator
    seeded by ``seed`` (then multiplied by ``scale`` and rounded)."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(lo), np.log(hi), nlambda))
    return np.round(n * scale).astype(np.uint64)


def torus_problem(n=256, nlambda=200, seed=1, npx=512, packet_scale=1.0) -> Problem:
    """Point source at the centre of the clumpy torus, 200 wavelengths
    0.09-10 micron, uneven packet counts per wavelength (1e5-2e7, log-uniform
    from the seed, times ``packet_scale``)."""
    grid = torus_grid(n, seed=seed)
    wl = powerlaw_wavelengths(nlambda, 0.09, 10.0)
    return Problem(
        name=f"torus{n}_l{nlambda}",
        grid=grid,
        source=Source(SRC_POINT, (0.0, 0.0, 0.0)),
        wl=wl,
        npk=uneven_packet_counts(nlambda, seed=seed, scale=packet_scale),
        instruments=galaxy_instruments(npx, fov=2.0),
        seed=seed,
    )


def beam_problem(grid: Grid, pos, direction, npackets=1, albedo=0.0, g=0.0,
                 instruments=None) -> Problem:
    return Problem(
        name="beam",
        grid=grid,
        source=Source(SRC_BEAM, tuple(float(v) for v in pos), tuple(float(v) for v in direction)),
        wl=single_wavelength(albedo=albedo, g=g),
        npk=np.array([npackets], dtype=np.uint64),
        instruments=list(instruments or []),
    )


# ----------------------------------------------------------------------------
# synthetic absorbed radiation fields (training and test inputs of the
# dust-emission step)
# ----------------------------------------------------------------------------
def absorbed_spectra(n, lam, seed=1, median=1.0, sigma_dex=1.0):
    """n absorbed spectra over the wavelengths ``lam`` [micron] and dust
    masses: a power law lambda^alpha (alpha uniform in [-2, 0.5]) attenuated by
    exp(-tau_V (lambda/0.55)^-1.2) (tau_V log-uniform in [1e-3, 1e2]), scaled so
    that the absorbed power per unit mass is log-normal with the given median
    and width in dex; masses log-uniform in [1e-7, 1e-4].  Returns
    (absorbed [n, len(lam)] float64, mass [n] float32)."""
    rng = np.random.default_rng(seed)
    lam = np.asarray(lam, dtype=np.float64)
    alpha = rng.uniform(-2.0, 0.5, n)
    tau_v = 10 ** rng.uniform(-3.0, 2.0, n)
    shape = lam[None, :] ** alpha[:, None] * np.exp(-tau_v[:, None] * (lam[None, :] / 0.55) ** -1.2)
    shape /= shape.sum(axis=1, keepdims=True)
    mass = (10 ** rng.uniform(-7.0, -4.0, n)).astype(np.float32)
    per_mass = median * 10 ** (sigma_dex * rng.normal(size=n))
    return shape * (per_mass * mass.astype(np.float64))[:, None], mass
