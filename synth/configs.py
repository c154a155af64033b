"""Workload definitions: the paper-scale configurations and small cases for tests.

A workload is a plain dict:

* ``geom``: kind, n (voxels per axis), h, angles (radians) or poses, nu, nv,
  pu, pv (bin pitch; radians for a curved detector), sod, sdd;
* ``part``: tiles per axis, view_blocks, det_blocks (du, dv);
* ``solver``: sampling (0 sequential, 1 uniform, 2 importance, 3 mixed),
  alpha, gamma, b, group_size, sync (0 column, 1 epoch), seed, theta_step;
* ``phantom``: number of shapes, seed; ``noise``: kind and level, seed;
* ``steps``: block steps of one solve.

Seeds: data seed 1709 + c, schedule seed 0x17090953 + c for configuration c.
The sizes follow the paper's simulations (Sec. III: 2D fan with 360 views,
2 x 2 volume blocks and 2 detector sub-areas; Sec. III-E: a 3D cone scan with
720 views and group size 90) scaled to the three workloads below.
"""
from __future__ import annotations

import math

import numpy as np

SCHED_SEED = 0x17090953


def _angles(n_views, span_deg):
    return np.deg2rad(np.arange(n_views) * (span_deg / n_views))


def parallel2d_64(steps_epochs: int = 50) -> dict:
    """2D parallel beam, 64^2 unit pixels, 90 views over [0, 180), 96 unit bins;
    2 view blocks x 2 x 2 tiles; uniform choice; 50 epochs (= 400 block steps)."""
    return dict(
        name="parallel2d_64_90x96_2x4_uniform",
        geom=dict(kind="parallel2d", n=(64, 64), h=1.0, angles=_angles(90, 180.0), nu=96,
                  nv=1, pu=1.0, pv=1.0, sod=0.0, sdd=0.0),
        part=dict(tiles=(2, 2), view_blocks=2, det_blocks=(1, 1)),
        solver=dict(sampling=1, alpha=1.0, gamma=1.0, b=2.0, group_size=1, sync=0,
                    seed=SCHED_SEED + 0, theta_step=1.0 / 40.0),
        phantom=dict(n_shapes=10, seed=1709 + 0),
        noise=dict(kind="gaussian", level=0.01, seed=1709 + 100),
        steps=steps_epochs * 8,
    )


def fan2d_512() -> dict:
    """2D fan beam, 512^2, 720 views over 360 deg, 768 curved bins, source at twice the
    image width from the centre; 8 view blocks x 4 x 4 tiles; density-weighted choice
    with alpha = 0.5; 200 block steps."""
    n = 512
    sod = 2.0 * n
    half_fan = math.asin(math.sqrt(2.0) * (n / 2) / sod)
    dg = 2.0 * half_fan / 768
    return dict(
        name="fan2d_512_720x768_8x16_importance",
        geom=dict(kind="fan2d_curved", n=(n, n), h=1.0, angles=_angles(720, 360.0), nu=768,
                  nv=1, pu=dg, pv=1.0, sod=sod, sdd=2.0 * sod),
        part=dict(tiles=(4, 4), view_blocks=8, det_blocks=(1, 1)),
        solver=dict(sampling=2, alpha=0.5, gamma=1.0, b=8.0, group_size=1, sync=0,
                    seed=SCHED_SEED + 1, theta_step=1.0 / 40.0),
        phantom=dict(n_shapes=20, seed=1709 + 1),
        noise=dict(kind="poisson", level=1e5, seed=1709 + 101),
        steps=200,
    )


def cone3d_256() -> dict:
    """3D cone beam, 256^3, 360 views on a circle, 384^2 pixels at pitch 2, SOD 512,
    SDD 1024; 360 single-view row blocks x 4x4x4 tiles; grouped choice with 30 views per
    group (12 groups per tile and epoch); one epoch = 768 group steps."""
    n = 256
    return dict(
        name="cone3d_256_360x384x384_360x64_g30",
        geom=dict(kind="cone3d", n=(n, n, n), h=1.0, angles=_angles(360, 360.0), nu=384,
                  nv=384, pu=2.0, pv=2.0, sod=2.0 * n, sdd=4.0 * n),
        part=dict(tiles=(4, 4, 4), view_blocks=360, det_blocks=(1, 1)),
        solver=dict(sampling=2, alpha=1.0, gamma=1.0, b=1.0, group_size=30, sync=0,
                    seed=SCHED_SEED + 2, theta_step=1.0 / 40.0),
        phantom=dict(n_shapes=30, seed=1709 + 2),
        noise=dict(kind="poisson", level=1e4, seed=1709 + 102),
        steps=768,
    )


def small_fan2d(n=96, views=60, nu=144, tiles=(3, 3), vb=4, du=2, curved=True, steps=40,
                sampling=2, group=1, alpha=0.5) -> dict:
    """A fan-beam case the oracle finishes in seconds, with ragged tiles."""
    sod = 2.0 * n
    half_fan = math.asin(math.sqrt(2.0) * (n / 2) / sod)
    if curved:
        pu = 2.0 * half_fan / nu
        kind = "fan2d_curved"
    else:
        pu = 2.0 * 2.0 * sod * math.tan(half_fan) / nu
        kind = "fan2d_flat"
    return dict(
        name="fan2d_%d_small" % n,
        geom=dict(kind=kind, n=(n, n), h=1.0, angles=_angles(views, 360.0), nu=nu, nv=1,
                  pu=pu, pv=1.0, sod=sod, sdd=2.0 * sod),
        part=dict(tiles=tiles, view_blocks=vb, det_blocks=(du, 1)),
        solver=dict(sampling=sampling, alpha=alpha, gamma=1.0, b=float(vb * du), group_size=group,
                    sync=0, seed=SCHED_SEED + 11, theta_step=1.0 / 40.0),
        phantom=dict(n_shapes=8, seed=1709 + 11),
        noise=dict(kind="poisson", level=1e5, seed=1709 + 111),
        steps=steps,
    )


def small_cone3d(n=24, views=24, nd=40, tiles=(2, 2, 3), group=4, steps=24, du=1, dv=1) -> dict:
    """A cone-beam case the oracle finishes in seconds, with ragged tiles."""
    return dict(
        name="cone3d_%d_small" % n,
        geom=dict(kind="cone3d", n=(n, n, n), h=1.0, angles=_angles(views, 360.0), nu=nd,
                  nv=nd, pu=2.0 * 1.5 * n / nd * 1.0, pv=2.0 * 1.5 * n / nd, sod=2.0 * n,
                  sdd=4.0 * n),
        part=dict(tiles=tiles, view_blocks=views, det_blocks=(du, dv)),
        solver=dict(sampling=2, alpha=1.0, gamma=1.0, b=1.0, group_size=group, sync=0,
                    seed=SCHED_SEED + 12, theta_step=1.0 / 40.0),
        phantom=dict(n_shapes=6, seed=1709 + 12),
        noise=dict(kind="poisson", level=1e4, seed=1709 + 112),
        steps=steps,
    )


def random_sphere_poses(n_views: int, radius: float, sdd: float, seed: int) -> np.ndarray:
    """Sec. III-E trajectory: source at radius r with random polar / azimuth angles,
    detector perpendicular to the source-centre line at distance sdd from the source.
    Returns (n_views, 12) = S, C, e_u, e_v."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((n_views, 12))
    for k in range(n_views):
        a = math.acos(1.0 - 2.0 * rng.random())
        b = 2.0 * math.pi * rng.random()
        S = radius * np.array([math.sin(a) * math.cos(b), math.sin(a) * math.sin(b), math.cos(a)])
        dc = -S / np.linalg.norm(S)
        C = S + sdd * dc
        ref = np.array([0.0, 0.0, 1.0]) if abs(dc[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
        eu = np.cross(ref, dc)
        eu /= np.linalg.norm(eu)
        ev = np.cross(dc, eu)
        out[k] = np.concatenate([S, C, eu, ev])
    return out


ALL = {"parallel2d_64": parallel2d_64, "fan2d_512": fan2d_512, "cone3d_256": cone3d_256}


def batch_fan2d(n_problems: int = 64, seed: int = 1709 + 3, n_range=(128, 1024),
                views_range=(60, 900), epochs: int = 3) -> list:
    """Many independent 2D fan-beam problems of seeded, uneven sizes (sparse-view
    included): n ~ U[128, 1024] pixels per side, views ~ U[60, 900], curved detector
    covering the circumscribed circle with 1.5 n bins, source at 2 n; 8 view blocks x
    4 x 4 tiles, density-weighted choice (alpha 0.5, b 8); a fixed number of epochs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_problems):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        views = int(rng.integers(views_range[0], views_range[1] + 1))
        nu = int(math.ceil(1.5 * n))
        sod = 2.0 * n
        half_fan = math.asin(math.sqrt(2.0) * (n / 2) / sod)
        vb = min(8, views)
        out.append(dict(
            name="batch_fan2d_%02d_%d_%dx%d" % (k, n, views, nu),
            geom=dict(kind="fan2d_curved", n=(n, n), h=1.0, angles=_angles(views, 360.0), nu=nu,
                      nv=1, pu=2.0 * half_fan / nu, pv=1.0, sod=sod, sdd=2.0 * sod),
            part=dict(tiles=(4, 4), view_blocks=vb, det_blocks=(1, 1)),
            solver=dict(sampling=2, alpha=0.5, gamma=1.0, b=float(vb), group_size=1, sync=0,
                        seed=SCHED_SEED + 100 + k, theta_step=1.0 / 40.0),
            phantom=dict(n_shapes=12, seed=1709 + 200 + k),
            noise=dict(kind="poisson", level=1e5, seed=1709 + 300 + k),
            steps=epochs * 16 * int(math.ceil(0.5 * vb)),
        ))
    return out


def cone3d_job(n: int, views: int, nd: int, tiles=(2, 2, 2), group: int = 30, epochs: int = 1,
               seed: int = 0, name: str = "") -> dict:
    """A circular cone-beam job: n^3 voxels, `views` views of nd^2 pixels at a pitch
    that covers the volume (SOD 2n, SDD 4n), single-view row blocks in groups."""
    pitch = 2.0 * 1.5 * n / nd
    groups = int(math.ceil(views / group))
    n_tiles = tiles[0] * tiles[1] * tiles[2]
    return dict(
        name=name or "cone3d_%d_%dx%d" % (n, views, nd),
        geom=dict(kind="cone3d", n=(n, n, n), h=1.0, angles=_angles(views, 360.0), nu=nd, nv=nd,
                  pu=pitch, pv=pitch, sod=2.0 * n, sdd=4.0 * n),
        part=dict(tiles=tiles, view_blocks=views, det_blocks=(1, 1)),
        solver=dict(sampling=2, alpha=1.0, gamma=1.0, b=1.0, group_size=group, sync=0,
                    seed=SCHED_SEED + 500 + seed, theta_step=1.0 / 40.0),
        phantom=dict(n_shapes=10, seed=1709 + 500 + seed),
        noise=dict(kind="poisson", level=1e4, seed=1709 + 600 + seed),
        steps=epochs * groups * n_tiles,
    )


def serving_jobs(n_jobs: int = 40, seed: int = 1709 + 4, small: bool = False) -> list:
    """A seeded mix of reconstruction requests: 2D fan beams of 256^2 .. 2048^2
    (64^2 .. 128^2 when small; 60 .. 720 views, 2 epochs) and 3D cone beams of
    128^3 .. 512^3 (24^3 .. 32^3 when small; 60 .. 180 views of (1.5 n)^2
    pixels, one epoch of groups of 30 views, 2^3 tiles up to 256^3 and 4^3
    tiles above), sizes log-uniform; one in eight a 100^3-volume job with 360
    views of 108^2 pixels (~4.2M rays, the paper's "a million unknowns, four
    million measurements" scale)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_jobs):
        kind = rng.random()
        size = rng.random()
        if kind < 0.45:
            lo, hi = (64, 128) if small else (256, 2048)
            n = int(round(lo * (hi / lo) ** size))
            views = int(rng.integers(60, 360 if small else 721))
            cfg = batch_fan2d(1, seed=seed * 1000 + k, n_range=(n, n), views_range=(views, views),
                              epochs=2)[0]
            cfg["name"] = "serve_fan2d_%02d_%d_%d" % (k, n, views)
        elif kind < 0.875 or small:
            lo, hi = (24, 32) if small else (128, 512)
            n = int(round(lo * (hi / lo) ** size))
            views = int(rng.integers(24, 60)) if small else int(rng.integers(60, 181))
            nd = int(1.5 * n)
            tiles = (2, 2, 2) if n <= 256 else (4, 4, 4)
            cfg = cone3d_job(n, views, nd, tiles=tiles, group=min(10 if small else 30, views), seed=k,
                             name="serve_cone3d_%02d_%d_%d" % (k, n, views))
        else:
            cfg = cone3d_job(100, 360, 108, group=30, seed=k, name="serve_cone3d_%02d_100_4M" % k)
        out.append(cfg)
    return out
