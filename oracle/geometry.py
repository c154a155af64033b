"""Scan geometries and the line of every measurement, in FP64 (oracle).

Test infrastructure only (see the package docstring).

The paper fixes the model y = Ax + e with A_i^j the length of ray i inside voxel
j (Sec. II-A), a point source whose detector is perpendicular to the line from
the source to the detector centre (Sec. II-D), a circular 2D fan trajectory
(Sec. III) and an arbitrary 3D trajectory (Sec. III-E).  It leaves the angle
origin, the rotation sense and the bin centring open; the readings used here
(and by every other part of this repository) are:

* the grid is centred on the origin: along axis a it spans
  [-n_a h / 2, n_a h / 2); voxel indices are row-major with x fastest;
* view v at angle theta: central direction d_c = (-cos t, -sin t[, 0]) (from
  the source towards the centre), detector axis e_u = (-sin t, cos t[, 0]) and,
  in 3D, e_v = (0, 0, 1); a cos or sin below 1e-12 is taken as exactly 0 (a
  view at a multiple of 90 degrees is axis-aligned; see ``axis_exact``);
* detector bin k (of n) has its centre at (k - (n-1)/2) * pitch along its axis;
* parallel beam: ray k is the line through s_k e_u with direction d_c;
* fan / cone with a flat detector: source S = sod * (cos t, sin t[, 0]), pixel
  centre P = S + sdd d_c + u e_u + v e_v, ray k is the line through S and P;
* fan with a curved detector (arc centred on the source): ray k leaves S in the
  direction cos(g_k) d_c + sin(g_k) e_u with g_k = (k - (n-1)/2) * pitch (radians);
* custom poses (3D): per view a source S, a detector centre C and unit axes
  e_u, e_v perpendicular to C - S; pixel centre P = C + u e_u + v e_v;
* measurements are ordered [view][v-bin][u-bin] (u fastest).

Parity: pinned through the analytic line integrals of ``synth`` (an independent
ray generator) in ``tests/test_oracle_siddon.py``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

KINDS = ("parallel2d", "fan2d_flat", "fan2d_curved", "cone3d", "custom3d")


@dataclass
class Grid:
    """Voxel grid of Sec. II-A: n voxels of edge h per axis, centred on 0."""

    n: tuple
    h: float = 1.0

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def lo(self) -> np.ndarray:
        return -0.5 * np.asarray(self.n, np.float64) * self.h

    @property
    def size(self) -> int:
        return int(np.prod(self.n))


@dataclass
class Geometry:
    """One scan: a grid, a detector and a list of views (Sec. II-D, Sec. III)."""

    kind: str
    n: tuple
    h: float = 1.0
    angles: np.ndarray = field(default_factory=lambda: np.zeros(0))
    nu: int = 1
    nv: int = 1
    pu: float = 1.0
    pv: float = 1.0
    sod: float = 0.0
    sdd: float = 0.0
    poses: np.ndarray | None = None  # custom3d: (n_views, 12) = S, C, e_u, e_v

    def __post_init__(self):
        assert self.kind in KINDS, self.kind
        self.n = tuple(int(v) for v in self.n)
        self.angles = np.asarray(self.angles, np.float64)
        if self.kind == "custom3d":
            self.poses = np.asarray(self.poses, np.float64).reshape(-1, 12)
        if self.kind in ("parallel2d", "fan2d_flat", "fan2d_curved"):
            assert len(self.n) == 2 and self.nv == 1
        else:
            assert len(self.n) == 3

    @property
    def grid(self) -> Grid:
        return Grid(self.n, self.h)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def n_views(self) -> int:
        if self.kind == "custom3d":
            return int(self.poses.shape[0])
        return int(self.angles.shape[0])

    @property
    def rays_per_view(self) -> int:
        return self.nu * self.nv

    @property
    def n_rays(self) -> int:
        return self.n_views * self.rays_per_view

    # ---- per-view frames -------------------------------------------------
    def frame(self, v: int):
        """(S, d_c, e_u, e_v, sdd) of view v in 3-vectors (z = 0 in 2D).

        For the parallel beam S is None.
        """
        if self.kind == "custom3d":
            p = self.poses[v]
            S, C, eu, ev = p[0:3], p[3:6], p[6:9], p[9:12]
            sdd = float(np.linalg.norm(C - S))
            return S.copy(), (C - S) / sdd, eu.copy(), ev.copy(), sdd
        t = float(self.angles[v])
        c, s = axis_exact(np.cos(t)), axis_exact(np.sin(t))
        dc = np.array([-c, -s, 0.0])
        eu = np.array([-s, c, 0.0])
        ev = np.array([0.0, 0.0, 1.0])
        if self.kind == "parallel2d":
            return None, dc, eu, ev, 0.0
        S = self.sod * np.array([c, s, 0.0])
        return S, dc, eu, ev, float(self.sdd)

    def bin_u(self, k):
        return (np.asarray(k, np.float64) - 0.5 * (self.nu - 1)) * self.pu

    def bin_v(self, k):
        return (np.asarray(k, np.float64) - 0.5 * (self.nv - 1)) * self.pv

    def view_rays(self, v: int, ku=None, kv=None):
        """Lines of view v as (origin, direction) arrays of shape (k, 3).

        ku / kv select bins (default: all, in [v-bin][u-bin] order).
        """
        if ku is None and kv is None:
            kvv, kuu = np.meshgrid(np.arange(self.nv), np.arange(self.nu), indexing="ij")
            ku, kv = kuu.reshape(-1), kvv.reshape(-1)
        ku = np.asarray(ku, np.float64).reshape(-1)
        kv = np.asarray(kv if kv is not None else np.zeros_like(ku), np.float64).reshape(-1)
        S, dc, eu, ev, sdd = self.frame(v)
        u = self.bin_u(ku)[:, None]
        w = self.bin_v(kv)[:, None]
        if self.kind == "parallel2d":
            org = u * eu[None, :]
            d = np.repeat(dc[None, :], ku.shape[0], axis=0)
        elif self.kind == "fan2d_curved":
            g = u  # pitch is an angle
            org = np.repeat(S[None, :], ku.shape[0], axis=0)
            d = np.cos(g) * dc[None, :] + np.sin(g) * eu[None, :]
        elif self.kind == "fan2d_flat":
            org = np.repeat(S[None, :], ku.shape[0], axis=0)
            d = sdd * dc[None, :] + u * eu[None, :]
        else:  # cone3d, custom3d
            org = np.repeat(S[None, :], ku.shape[0], axis=0)
            d = sdd * dc[None, :] + u * eu[None, :] + w * ev[None, :]
        return org, d

    def rays(self, ray_ids=None):
        """(origin, direction) of the given global ray indices (default: all)."""
        if ray_ids is None:
            ray_ids = np.arange(self.n_rays)
        ray_ids = np.asarray(ray_ids, np.int64).reshape(-1)
        rpv = self.rays_per_view
        views = ray_ids // rpv
        within = ray_ids % rpv
        org = np.zeros((ray_ids.shape[0], 3))
        d = np.zeros((ray_ids.shape[0], 3))
        for v in np.unique(views):
            sel = views == v
            o, dd = self.view_rays(int(v), within[sel] % self.nu, within[sel] // self.nu)
            org[sel] = o
            d[sel] = dd
        return org, d

    # ---- detector coordinates (used by the importance table) ------------
    def detector_coords(self, v: int, pts: np.ndarray):
        """Continuous bin coordinates (w_u, w_v) of world points seen from view v.

        Bin k covers [k, k+1) in these coordinates, so the bin centre is k + 1/2.
        """
        pts = np.asarray(pts, np.float64).reshape(-1, 3)
        S, dc, eu, ev, sdd = self.frame(v)
        if self.kind == "parallel2d":
            wu = pts @ eu / self.pu + 0.5 * self.nu
            return wu, np.full_like(wu, 0.5)
        rel = pts - S[None, :]
        depth = rel @ dc
        if self.kind == "fan2d_curved":
            g = np.arctan2(rel @ eu, depth)
            return g / self.pu + 0.5 * self.nu, np.full(pts.shape[0], 0.5)
        lam = sdd / depth
        wu = lam * (rel @ eu) / self.pu + 0.5 * self.nu
        if self.dim == 2:
            return wu, np.full_like(wu, 0.5)
        wv = lam * (rel @ ev) / self.pv + 0.5 * self.nv
        return wu, wv


def axis_exact(v: float) -> float:
    """A cosine or sine of a view angle below 1e-12 in magnitude is exactly 0.

    Reading: a view at a multiple of 90 degrees is axis-aligned (cos(pi/2)
    evaluates to 6e-17); a 1e-16 tilt would move the point where such a line
    crosses a voxel face anywhere along it, which no finite precision can place.
    """
    return 0.0 if abs(v) < 1e-12 else float(v)


def uniform_angles(n_views: int, span_deg: float, start_deg: float = 0.0) -> np.ndarray:
    """theta_v = start + v * span / n_views, in radians."""
    return np.deg2rad(start_deg + np.arange(n_views) * (span_deg / n_views))
