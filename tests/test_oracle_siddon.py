"""Pins of the FP64 Siddon oracle (Sec. II-A: A_i^j = length of ray i in voxel j).

Each test checks the oracle against something other than itself: a brute-force
slab clip of every (ray, voxel) pair, closed forms for axis-aligned and
diagonal rays, the chord of the grid's bounding box, and exact line integrals
of ellipses / ellipsoids computed by ``synth`` from its own ray generator.
"""
import math

import numpy as np
import pytest

from oracle import siddon
from oracle.geometry import Geometry, Grid, uniform_angles
from synth import phantom as PH


def brute_force(grid: Grid, org, d):
    """Dense A by Liang-Barsky clipping of each line against each voxel box."""
    org = np.asarray(org, float).reshape(-1, 3)
    d = np.asarray(d, float).reshape(-1, 3)
    dim = grid.dim
    n = grid.n
    lo = grid.lo
    h = grid.h
    A = np.zeros((org.shape[0], grid.size))
    idx = np.stack(np.meshgrid(*[np.arange(k) for k in n], indexing="ij"), -1).reshape(-1, dim)
    for i in range(org.shape[0]):
        dn = np.linalg.norm(d[i, :dim])
        for v in idx:
            t0, t1 = -np.inf, np.inf
            ok = True
            for a in range(dim):
                b0 = lo[a] + v[a] * h
                b1 = b0 + h
                if d[i, a] == 0.0:
                    if not (b0 <= org[i, a] < b1):
                        ok = False
                    continue
                ta = (b0 - org[i, a]) / d[i, a]
                tb = (b1 - org[i, a]) / d[i, a]
                t0 = max(t0, min(ta, tb))
                t1 = min(t1, max(ta, tb))
            if ok and t1 > t0:
                L = (t1 - t0) * dn
                if L > 1e-12 * h:
                    col = v[0] + n[0] * v[1] + (n[0] * n[1] * v[2] if dim == 3 else 0)
                    A[i, col] = L
    return A


def _geoms_small():
    rng = np.random.default_rng(5)
    ang = rng.uniform(0, 2 * np.pi, 3)
    out = [
        Geometry("parallel2d", (7, 6), 1.0, ang, nu=9, pu=0.83),
        Geometry("fan2d_flat", (6, 7), 0.7, ang, nu=10, pu=0.9, sod=14.0, sdd=25.0),
        Geometry("fan2d_curved", (8, 8), 1.0, ang, nu=11, pu=0.07, sod=20.0, sdd=40.0),
        Geometry("cone3d", (5, 4, 6), 1.0, ang, nu=6, nv=5, pu=1.3, pv=1.1, sod=15.0, sdd=30.0),
    ]
    return out


@pytest.mark.parametrize("k", range(4))
def test_alpha_merge_equals_brute_force(k):
    g = _geoms_small()[k]
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d).toarray()
    B = brute_force(g.grid, org, d)
    assert A.shape == B.shape
    assert np.abs(A).sum() > 0
    assert np.max(np.abs(A - B)) <= 1e-13 * max(1.0, g.h)


def test_custom_random_sphere_brute_force():
    from synth.configs import random_sphere_poses
    poses = random_sphere_poses(4, 12.0, 24.0, seed=3)
    g = Geometry("custom3d", (4, 5, 4), 1.0, nu=5, nv=4, pu=1.5, pv=1.5, poses=poses)
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d).toarray()
    B = brute_force(g.grid, org, d)
    assert np.abs(A).sum() > 0
    assert np.max(np.abs(A - B)) <= 1e-13


def test_axis_aligned_rays_through_pixel_centres():
    """theta = 0: horizontal rays through pixel-centre rows; every entry equals h and
    a ray sum equals the sum of one image row."""
    n = 16
    g = Geometry("parallel2d", (n, n), 0.5, np.array([0.0]), nu=n, pu=0.5)
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d)
    vals = A.data
    assert vals.size == n * n
    assert np.all(vals == 0.5)
    x = np.random.default_rng(0).random(n * n)
    rowsum = x.reshape(n, n).sum(axis=1) * 0.5
    np.testing.assert_allclose(A @ x, rowsum, rtol=1e-14)


def test_diagonal_rays_through_corners():
    """A 45-degree line through grid vertices crosses each diagonal voxel with length
    sqrt(2) h and touches its neighbours only at corners (structural zeros)."""
    n, h = 10, 1.0
    grid = Grid((n, n), h)
    org = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    d = np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 0.0]])
    A = siddon.system_matrix(grid, org, d)
    row0 = A.getrow(0)
    assert row0.nnz == n
    np.testing.assert_allclose(row0.data, math.sqrt(2.0) * h, rtol=0, atol=1e-13)
    cols = np.sort(row0.indices)
    np.testing.assert_array_equal(cols, [i * n + i for i in range(n)])
    row1 = A.getrow(1)
    assert row1.nnz == n - 1


def test_line_on_plane_goes_to_plus_side():
    """Half-open voxels: a line lying on the plane x = 0 belongs to the column x >= 0."""
    grid = Grid((4, 4), 1.0)
    A = siddon.system_matrix(grid, np.array([[0.0, -10.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    cols = np.sort(A.indices)
    np.testing.assert_array_equal(cols, [2, 6, 10, 14])
    np.testing.assert_allclose(A.data, 1.0)


def _bbox_chord(grid, o, d):
    lo = grid.lo
    hi = lo + np.asarray(grid.n) * grid.h
    t0, t1 = -np.inf, np.inf
    for a in range(grid.dim):
        if d[a] == 0:
            if not (lo[a] <= o[a] < hi[a]):
                return 0.0
            continue
        ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0) * np.linalg.norm(d[:grid.dim])


@pytest.mark.parametrize("kind", ["fan2d_curved", "cone3d"])
def test_row_sum_is_bounding_box_chord(kind):
    if kind == "fan2d_curved":
        g = Geometry(kind, (40, 33), 1.0, uniform_angles(7, 360), nu=50, pu=0.03, sod=80, sdd=160)
    else:
        g = Geometry(kind, (12, 10, 14), 1.0, uniform_angles(5, 360), nu=20, nv=18, pu=2, pv=2,
                     sod=30, sdd=60)
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d)
    sums = np.asarray(A.sum(axis=1)).ravel()
    ref = np.array([_bbox_chord(g.grid, org[i], d[i]) for i in range(org.shape[0])])
    assert ref.max() > 0
    np.testing.assert_allclose(sums, ref, rtol=0, atol=1e-10)


def test_ellipse_line_integrals_converge():
    """A x_h -> exact line integrals of the phantom as h -> 0, with an O(h) trend.

    The exact values come from synth's own rays (independent of the oracle's
    geometry code), so a wrong angle origin, rotation sense or bin centre fails."""
    spec = dict(kind="fan2d_curved", angles=uniform_angles(12, 360), nu=64, pu=0.012,
                sod=64.0, sdd=128.0)
    width = 32.0
    ph = PH.make_phantom(2, 5, width / 2, seed=11)
    org_s, d_s = PH.rays_of(spec)
    exact = PH.line_integrals(ph, org_s, d_s)
    errs = []
    for n in (32, 64, 128):
        h = width / n
        g = Geometry("fan2d_curved", (n, n), h, spec["angles"], nu=64, pu=0.012, sod=64.0,
                     sdd=128.0)
        xh = PH.pixelize(ph, (n, n), h, sub=8)
        org, d = g.rays()
        A = siddon.system_matrix(g.grid, org, d)
        errs.append(np.sqrt(np.mean((A @ xh - exact) ** 2)) / np.sqrt(np.mean(exact ** 2)))
    # O(h): each halving of h at least ~halves the error (measured 0.058, 0.032, 0.016)
    assert errs[0] < 0.1
    assert errs[1] < 0.7 * errs[0] and errs[2] < 0.7 * errs[1]
    assert errs[2] < 0.025
    # the test can tell a mirrored scan apart: the opposite rotation sense is far off
    spec_m = dict(spec, angles=-spec["angles"])
    om, dm = PH.rays_of(spec_m)
    wrong = PH.line_integrals(ph, om, dm)
    assert np.sqrt(np.mean((A @ xh - wrong) ** 2)) / np.sqrt(np.mean(exact ** 2)) > 10 * errs[2]


def test_ellipsoid_line_integrals_converge():
    spec = dict(kind="cone3d", angles=uniform_angles(4, 360), nu=24, nv=24, pu=1.6, pv=1.6,
                sod=40.0, sdd=80.0)
    width = 16.0
    ph = PH.make_phantom(3, 4, width / 2, seed=12)
    org_s, d_s = PH.rays_of(spec)
    exact = PH.line_integrals(ph, org_s, d_s)
    errs = []
    for n in (16, 32):
        h = width / n
        g = Geometry("cone3d", (n, n, n), h, spec["angles"], nu=24, nv=24, pu=1.6, pv=1.6,
                     sod=40.0, sdd=80.0)
        xh = PH.pixelize(ph, (n, n, n), h, sub=4)
        org, d = g.rays()
        A = siddon.system_matrix(g.grid, org, d)
        errs.append(np.sqrt(np.mean((A @ xh - exact) ** 2)) / np.sqrt(np.mean(exact ** 2)))
    # O(h): measured 0.27 at n = 16 and 0.13 at n = 32 (0.06 at n = 64)
    assert errs[0] < 0.35
    assert errs[1] < 0.6 * errs[0]


def test_parallel_projection_of_disc():
    """A centred disc of radius a and value 1: the parallel projection at offset s is
    2 sqrt(a^2 - s^2) for every angle (checks bin centring of the oracle's rays)."""
    n, h, a = 128, 0.25, 12.0
    ph = dict(dim=2, centres=np.zeros((1, 3)), axes=np.array([[a, a, 1.0]]),
              rot=np.eye(3)[None], values=np.array([1.0]))
    ang = uniform_angles(6, 180)
    g = Geometry("parallel2d", (n, n), h, ang, nu=40, pu=0.7)
    xh = PH.pixelize(ph, (n, n), h, sub=8)
    org, d = g.rays()
    p = siddon.system_matrix(g.grid, org, d) @ xh
    s = g.bin_u(np.arange(40))
    ref = np.tile(2 * np.sqrt(np.maximum(a * a - s * s, 0)), 6)
    # pixelisation error concentrates on near-tangent rays; measured 0.6% RMS
    assert np.sqrt(np.mean((p - ref) ** 2)) < 0.01 * np.sqrt(np.mean(ref ** 2))
    # a half-bin shift of the bin centres would be far worse
    ref_shift = np.tile(2 * np.sqrt(np.maximum(a * a - (s + 0.35) ** 2, 0)), 6)
    assert np.sqrt(np.mean((p - ref_shift) ** 2)) > 3 * np.sqrt(np.mean((p - ref) ** 2))


def _rel_rms(a, b):
    return np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2))


def test_flat_fan_line_integrals_converge():
    """The flat-detector fan (the Sec. III scan's detector) against exact line
    integrals along synth's own rays: O(h) convergence, and a mirrored detector
    (u axis reversed) or the opposite rotation sense is far off."""
    spec = dict(kind="fan2d_flat", angles=uniform_angles(10, 360) + 0.1, nu=48, pu=0.9,
                sod=40.0, sdd=80.0)
    width = 24.0
    ph = PH.make_phantom(2, 5, width / 2, seed=21)
    exact = PH.line_integrals(ph, *PH.rays_of(spec))
    errs = []
    for n in (24, 48, 96):
        h = width / n
        g = Geometry("fan2d_flat", (n, n), h, spec["angles"], nu=48, pu=0.9, sod=40.0, sdd=80.0)
        xh = PH.pixelize(ph, (n, n), h, sub=8)
        A = siddon.system_matrix(g.grid, *g.rays())
        errs.append(_rel_rms(A @ xh, exact))
    assert errs[0] < 0.1
    assert errs[1] < 0.7 * errs[0] and errs[2] < 0.7 * errs[1]
    p = A @ xh
    mirrored = PH.line_integrals(ph, *PH.rays_of(dict(spec, pu=-spec["pu"])))
    assert _rel_rms(p, mirrored) > 10 * errs[2]
    reversed_sense = PH.line_integrals(ph, *PH.rays_of(dict(spec, angles=-spec["angles"])))
    assert _rel_rms(p, reversed_sense) > 10 * errs[2]


def test_custom_pose_line_integrals_converge():
    """Arbitrary per-view poses (Sec. III-E, random spherical orbit): the oracle's
    lines through C + u e_u + v e_v from S against exact line integrals along
    synth's own rays of the same poses; a detector with e_u mirrored, or with
    e_u and e_v swapped, is far off."""
    from synth.configs import random_sphere_poses
    poses = random_sphere_poses(6, 30.0, 60.0, seed=5)
    spec = dict(kind="custom3d", poses=poses, nu=20, nv=16, pu=1.7, pv=1.9)
    width = 16.0
    ph = PH.make_phantom(3, 4, width / 2, seed=22)
    exact = PH.line_integrals(ph, *PH.rays_of(spec))
    errs = []
    for n in (16, 32):
        h = width / n
        g = Geometry("custom3d", (n, n, n), h, nu=20, nv=16, pu=1.7, pv=1.9, poses=poses)
        xh = PH.pixelize(ph, (n, n, n), h, sub=4)
        A = siddon.system_matrix(g.grid, *g.rays())
        errs.append(_rel_rms(A @ xh, exact))
    assert errs[0] < 0.35
    assert errs[1] < 0.6 * errs[0]
    p = A @ xh
    mir = poses.copy()
    mir[:, 6:9] *= -1.0
    assert _rel_rms(p, PH.line_integrals(ph, *PH.rays_of(dict(spec, poses=mir)))) > 4 * errs[1]
    swp = poses.copy()
    swp[:, 6:9], swp[:, 9:12] = poses[:, 9:12], poses[:, 6:9]
    assert _rel_rms(p, PH.line_integrals(ph, *PH.rays_of(dict(spec, poses=swp)))) > 4 * errs[1]
