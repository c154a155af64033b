"""Importance table P(I, J) = P_S / P_T (Sec. II-C, Alg. 3), FP64.

Test infrastructure only (see the package docstring).

Alg. 3 defines P_S as the area of the projection of the selected volume block J
that falls on the selected detector sub-area I, and P_T as the total projection
area of J on the whole detector over the whole trajectory.  The readings used:

* "projection of J" in view v is the exact shadow of the cuboid on the
  detector: in 2D the interval between the extreme corner coordinates, in 3D
  the convex hull of the eight projected corners;
* areas are measured in detector-bin units (bin k covers [k, k+1));
* a row block I with several views sums the per-view overlaps, so a group
  I_g = union of row blocks has P_S(I_g, J) = sum of the members' P_S and
  beta = b * P_S(I_g, J) / P_T(J) grows with the group, as Sec. III-B notes;
* P_T(J) = 0 (a tile no ray sees) gives P(., J) = 0;
* an overlap below 1e-9 bin units counts as none: a shadow edge that falls
  exactly on a sub-area boundary otherwise leaves a rounding sliver whose sign
  decides whether the block can be drawn at all.

Pinned in ``tests/test_oracle_ptable.py`` by the parallel-beam closed form of
the shadow width, sum_I P(I, J) = 1, symmetry and hand-computed hull cases.
"""
from __future__ import annotations

import numpy as np

from .blocks import Partition

SLIVER = 1e-9  # overlaps below this many bin units count as zero


def _tile_corners(part: Partition, j: int) -> np.ndarray:
    g = part.geom
    lo, hi = part.tile_box(j)
    glo = g.grid.lo
    wlo = [glo[a] + lo[a] * g.h for a in range(g.dim)]
    whi = [glo[a] + hi[a] * g.h for a in range(g.dim)]
    if g.dim == 2:
        return np.array([[x, y, 0.0] for x in (wlo[0], whi[0]) for y in (wlo[1], whi[1])])
    return np.array([[x, y, z] for x in (wlo[0], whi[0]) for y in (wlo[1], whi[1])
                     for z in (wlo[2], whi[2])])


def convex_hull(pts: np.ndarray) -> np.ndarray:
    """Counter-clockwise convex hull of 2D points (Andrew's monotone chain)."""
    p = sorted(set((float(a), float(b)) for a, b in pts))
    if len(p) <= 2:
        return np.array(p)

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])

    lower, upper = [], []
    for q in p:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], q) <= 0:
            lower.pop()
        lower.append(q)
    for q in reversed(p):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], q) <= 0:
            upper.pop()
        upper.append(q)
    return np.array(lower[:-1] + upper[:-1])


def clip_polygon_rect(poly: np.ndarray, x0, x1, y0, y1) -> np.ndarray:
    """Sutherland-Hodgman clip of a convex polygon against [x0,x1] x [y0,y1]."""
    def clip(points, inside, intersect):
        out = []
        n = len(points)
        for k in range(n):
            cur, prev = points[k], points[k - 1]
            if inside(cur):
                if not inside(prev):
                    out.append(intersect(prev, cur))
                out.append(cur)
            elif inside(prev):
                out.append(intersect(prev, cur))
        return out

    def ix(xc):
        return lambda a, b: (xc, a[1] + (b[1] - a[1]) * (xc - a[0]) / (b[0] - a[0]))

    def iy(yc):
        return lambda a, b: (a[0] + (b[0] - a[0]) * (yc - a[1]) / (b[1] - a[1]), yc)

    pts = [tuple(q) for q in poly]
    for inside, inter in ((lambda q: q[0] >= x0, ix(x0)), (lambda q: q[0] <= x1, ix(x1)),
                          (lambda q: q[1] >= y0, iy(y0)), (lambda q: q[1] <= y1, iy(y1))):
        if not pts:
            break
        pts = clip(pts, inside, inter)
    return np.array(pts)


def polygon_area(poly: np.ndarray) -> float:
    """Shoelace area of a simple polygon."""
    if len(poly) < 3:
        return 0.0
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * abs(float(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1))))


def shadow(part: Partition, v: int, j: int):
    """Shadow of tile j in view v: an interval (2D) or a convex polygon (3D)."""
    g = part.geom
    wu, wv = g.detector_coords(v, _tile_corners(part, j))
    if g.dim == 2:
        return float(wu.min()), float(wu.max())
    return convex_hull(np.stack([wu, wv], axis=1))


def overlap(part: Partition, v: int, j: int, u0, u1, v0, v1) -> float:
    """Area of the shadow of tile j in view v inside [u0,u1) x [v0,v1) (bin units)."""
    s = shadow(part, v, j)
    if part.geom.dim == 2:
        lo, hi = s
        a = max(0.0, min(hi, u1) - max(lo, u0))
    else:
        a = polygon_area(clip_polygon_rect(s, u0, u1, v0, v1))
    return a if a > SLIVER else 0.0


def shadow_tables(part: Partition):
    """(P_S, P_T): P_S[i, j] over row blocks, P_T[j] over the whole detector."""
    g = part.geom
    m, n = part.n_row_blocks, part.n_col_blocks
    PS = np.zeros((m, n))
    PT = np.zeros(n)
    for j in range(n):
        for v in range(g.n_views):
            PT[j] += overlap(part, v, j, 0, g.nu, 0, g.nv)
        for i in range(m):
            u0, u1, v0, v1 = part.row_block_subrect(i)
            PS[i, j] = sum(overlap(part, int(v), j, u0, u1, v0, v1)
                           for v in part.row_block_views(i))
    return PS, PT


def probability_table(part: Partition) -> np.ndarray:
    """P(I, J) = P_S(I, J) / P_T(J) as an (m, n) array (Alg. 3, initialisation)."""
    PS, PT = shadow_tables(part)
    P = np.zeros_like(PS)
    nz = PT > 0
    P[:, nz] = PS[:, nz] / PT[nz][None, :]
    return P
