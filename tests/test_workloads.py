"""The synthetic inputs match the recipe they are described by: the disk's
face-on optical depth through its centre, the smooth torus's equatorial
optical depth, the sphere's volume-weighted extinction, and the uneven
packet counts' range (column sums over the generated grids)."""
import math

import numpy as np

from paper_1705_04702_gb300 import workloads as W


def test_disk_face_on_optical_depth_is_one():
    """kr0 = tau_face / (2 h_z): the column through (near) the centre sums to
    e^{-R/h_R} (1 - e^{-3/h_z}) with tau_face = 1, up to the z sampling."""
    g = W.disk_grid(64, nxyz=(64, 64, 256))
    dz = (g.bbox[5] - g.bbox[4]) / g.nz
    col = g.kr[:, 31, 31].astype(np.float64).sum() * dz
    R = math.hypot(*[(31 + 0.5) * (48.0 / 64) - 24.0] * 2)
    assert abs(col - math.exp(-R / 6.0) * (1 - math.exp(-12.0))) < 2e-3


def test_torus_normalisation_and_clumps():
    """The smooth torus is kr0 r^-1 e^{-6 |cos theta|} with kr0 = 10 / ln 20,
    so that the continuum equatorial optical depth from r = 0.05 to 1 is 10;
    with clumps, about 5% of the dusty cells carry 100x the smooth value."""
    smooth = W.torus_grid(64, clump_fraction=0.0)
    clumpy = W.torus_grid(64)
    d = 2.0 / 64
    kr0 = 10.0 / math.log(20.0)
    assert abs(kr0 * math.log(1.0 / 0.05) - 10.0) < 1e-12
    for iz, iy, ix in ((32, 32, 50), (33, 40, 45), (30, 20, 60)):
        x, y, z = (-1.0 + (np.array([ix, iy, iz]) + 0.5) * d)
        r = math.sqrt(x * x + y * y + z * z)
        expect = kr0 / r * math.exp(-6.0 * abs(z) / r)
        assert smooth.kr[iz, iy, ix] == np.float32(expect)
    dusty = smooth.kr > 0
    ratio = clumpy.kr[dusty] / smooth.kr[dusty]
    assert set(np.unique(np.round(ratio, 3))) <= {1.0, 100.0}
    assert abs((ratio > 1).mean() - 0.05) < 0.005


def test_sphere_extinction_is_volume_weighted():
    g = W.sphere_grid(32)
    vol = (2.0 / 32) ** 3
    assert abs(g.kr.astype(np.float64).sum() * vol - 4.0 / 3.0 * math.pi) < 0.02


def test_uneven_packet_counts_range():
    n = W.uneven_packet_counts(200, seed=1)
    assert n.min() >= 1e5 and n.max() <= 2e7
    assert 5e8 < n.sum() < 1e9
