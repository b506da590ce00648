"""The drop-impact measures (cavity depth and crown inner diameter in the
centre cross-section) on phi fields whose answers are known by construction:
a flat pool, a pool with a hemispherical cavity of radius R (depth -R / D,
diameter 2 R / D at the initial surface), the same with a droplet in the air
right above the cavity bottom (which hides the bottom from a scan coming down
from the top), and a cavity off the measuring plane (which must not be seen).
"""
import numpy as np

from paper_2206_11637_gb300 import impact as I
from paper_2206_11637_gb300 import workloads as W


def pool_with_cavity(R, xi=4.0, offset_x=0.0, droplet=False):
    p = W.Params(81, 80, 81, (0, 0, 1, 1, 0, 0), 1.0, 1e-3, 0.01, 0.01, 1e-4, 0.03, xi)
    y0 = 39.5
    x, y, z = W.coords(p)
    # the surface around the cavity stands 3 cells above y0, as a crown does,
    # so the row y = y0 is liquid outside the cavity
    pool = W.tanh_profile(y - (y0 + 3.0 if R > 0 else y0), xi)
    if R > 0:
        cav = W.sphere(p, (40.0 + offset_x, y0, 40.0), R, heavy_inside=True)
        pool = np.minimum(pool, 1.0 - cav)
    if droplet:
        pool = np.maximum(pool, W.sphere(p, (40.0, y0 + 25.0, 40.0), 4.0, heavy_inside=True))
    return pool, y0


def test_flat_pool():
    phi, y0 = pool_with_cavity(0.0)
    assert abs(I.cavity_depth(phi, y0, 20.0)) < 1e-9
    assert I.crown_diameter(phi, y0, 20.0) == 0.0


def test_hemispherical_cavity():
    for R in (10.0, 16.0):
        phi, y0 = pool_with_cavity(R)
        D = 20.0
        assert abs(I.cavity_depth(phi, y0, D) + R / D) < 0.01
        assert abs(I.crown_diameter(phi, y0, D) - 2 * R / D) < 0.01


def test_droplet_above_does_not_hide_the_cavity():
    phi, y0 = pool_with_cavity(12.0, droplet=True)
    assert abs(I.cavity_depth(phi, y0, 20.0) + 12.0 / 20.0) < 0.01


def test_cavity_off_the_plane_is_not_seen():
    phi, y0 = pool_with_cavity(8.0, offset_x=25.0)
    # only the raised surface (3 cells above y0) is in the plane
    assert abs(I.cavity_depth(phi, y0, 20.0) - 3.0 / 20.0) < 1e-3
