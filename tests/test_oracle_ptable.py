"""Pins of the oracle's importance table P(I, J) = P_S / P_T (Sec. II-C, Alg. 3)."""
import math

import numpy as np
import pytest

from oracle import ptable
from oracle.blocks import Partition
from oracle.geometry import Geometry, uniform_angles


def test_parallel_shadow_width_closed_form():
    """A W x H tile seen along d_c = -(cos t, sin t) casts a shadow of width
    W |sin t| + H |cos t| on the axis e_u = (-sin t, cos t)."""
    ang = np.deg2rad([0.0, 17.0, 45.0, 90.0, 133.0])
    g = Geometry("parallel2d", (40, 30), 1.0, ang, nu=200, pu=0.5)
    part = Partition(g, tiles=(2, 3))
    for j in range(part.n_col_blocks):
        lo, hi = part.tile_box(j)
        W, H = hi[0] - lo[0], hi[1] - lo[1]
        for v, t in enumerate(ang):
            a, b = ptable.shadow(part, v, j)
            np.testing.assert_allclose((b - a) * 0.5, W * abs(math.sin(t)) + H * abs(math.cos(t)),
                                       rtol=1e-12)


def test_probabilities_sum_to_one_over_a_covering_partition():
    g = Geometry("fan2d_curved", (48, 48), 1.0, uniform_angles(36, 360), nu=120, pu=0.025,
                 sod=96, sdd=192)
    part = Partition(g, tiles=(3, 2), view_blocks=4, det_blocks=(3, 1))
    P = ptable.probability_table(part)
    assert P.shape == (12, 6)
    assert np.all(P >= 0)
    np.testing.assert_allclose(P.sum(axis=0), 1.0, rtol=1e-12)


def test_symmetric_tiles_have_mirrored_tables():
    """Parallel beam over [0, 180) with 2 view blocks: the two tiles on a diagonal of a
    2 x 2 split are related by a 180-degree rotation, which maps each view onto itself
    with the detector reversed; so P of the mirrored sub-area is equal."""
    g = Geometry("parallel2d", (32, 32), 1.0, uniform_angles(30, 180), nu=48, pu=1.0)
    part = Partition(g, tiles=(2, 2), view_blocks=2, det_blocks=(2, 1))
    P = ptable.probability_table(part)
    # row block = (vb, du); rotation by 180 deg swaps du 0 <-> 1, keeps vb; tile 0 <-> 3
    for vb in range(2):
        for du in range(2):
            i = vb * 2 + du
            i_m = vb * 2 + (1 - du)
            np.testing.assert_allclose(P[i, 0], P[i_m, 3], rtol=1e-12)
            np.testing.assert_allclose(P[i, 1], P[i_m, 2], rtol=1e-12)


def test_cone_shadow_area_closed_form():
    """theta = 0, cube [-a, a]^3 centred on the axis: the hull of the projected corners
    is the square of the near face, side 2 a sdd / (sod - a) on the detector."""
    a = 4.0
    g = Geometry("cone3d", (8, 8, 8), 1.0, np.array([0.0]), nu=64, nv=64, pu=0.5, pv=0.5,
                 sod=20.0, sdd=40.0)
    part = Partition(g, tiles=(1, 1, 1), view_blocks=1)
    side = 2 * a * 40.0 / (20.0 - a) / 0.5
    full = ptable.overlap(part, 0, 0, 0, 64, 0, 64)
    np.testing.assert_allclose(full, side * side, rtol=1e-12)
    # a quarter sub-area sees exactly a quarter of the centred square
    q = ptable.overlap(part, 0, 0, 0, 32, 0, 32)
    np.testing.assert_allclose(q, side * side / 4, rtol=1e-12)


def test_hull_and_clip_helpers():
    pts = np.array([[0, 0], [2, 0], [2, 2], [0, 2], [1, 1], [1, 0]], float)
    hull = ptable.convex_hull(pts)
    assert len(hull) == 4
    assert ptable.polygon_area(hull) == pytest.approx(4.0)
    tri = np.array([[0, 0], [4, 0], [0, 4]], float)
    clipped = ptable.clip_polygon_rect(tri, 1, 3, 0, 2)
    # area of the triangle x + y <= 4 inside [1,3] x [0,2]: 4 - 0.5 = 3.5
    assert ptable.polygon_area(clipped) == pytest.approx(3.5)


def test_tile_outside_every_sub_area_has_zero_probability():
    g = Geometry("parallel2d", (40, 40), 1.0, np.array([0.0]), nu=80, pu=1.0)
    part = Partition(g, tiles=(1, 4), view_blocks=1, det_blocks=(4, 1))
    P = ptable.probability_table(part)
    # at theta = 0 tile rows map one-to-one onto the central 40 bins: tile k (y range
    # [10k - 20, 10k - 10)) falls in bins [10k + 20, 10k + 30) = sub-area 1 or 2 only
    assert P[0].sum() == 0 and P[3].sum() == 0
    np.testing.assert_allclose(P.sum(axis=0), 1.0)
