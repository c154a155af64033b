"""Seeded ellipse / ellipsoid phantoms, their exact line integrals and noise.

Recipe (the paper's phantoms are not printed, so these stand in for them):

* R = half the grid width; centres uniform in the disc / ball of radius 0.6 R;
  semi-axes uniform in [0.05 R, 0.45 R]; 2D orientation uniform in [0, pi), 3D
  orientation from a uniform random unit quaternion; attenuation uniform in
  [0, 1]; shapes add up; a shape is redrawn unless |centre| + largest semi-axis
  <= 0.95 R (so it lies inside the inscribed circle / sphere);
* clean data are exact line integrals (chord length through each shape times its
  value, from the line-quadric intersection);
* Gaussian noise: sigma = 1% of max(y_clean);
* Poisson noise at N0 photons per ray: the phantom is first scaled so that
  max(y_clean) = 4 (the scale is returned), then k ~ Poisson(N0 exp(-y)) and
  y = ln(N0 / max(k, 1));
* every random number comes from numpy's PCG64 with the given seed.

Line integrals can be evaluated with numpy (CPU) or torch (any device), both in
FP64; they use this module's own ray generator (``rays_of``).
"""
from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# phantom parameters
# ---------------------------------------------------------------------------
def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Rotation matrix of a uniformly random unit quaternion (Shoemake 1992)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def make_phantom(dim: int, n_shapes: int, radius: float, seed: int) -> dict:
    """Random shapes: dict(centres (k,3), axes (k,3), rot (k,3,3), values (k,))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C, AX, ROT, VAL = [], [], [], []
    while len(C) < n_shapes:
        if dim == 2:
            rr = 0.6 * radius * math.sqrt(rng.random())
            ph = 2 * math.pi * rng.random()
            c = np.array([rr * math.cos(ph), rr * math.sin(ph), 0.0])
            ax = np.array([rng.uniform(0.05, 0.45) * radius, rng.uniform(0.05, 0.45) * radius, 1.0])
            a = math.pi * rng.random()
            rot = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0],
                            [0.0, 0.0, 1.0]])
            big = max(ax[0], ax[1])
        else:
            while True:
                c = rng.uniform(-0.6 * radius, 0.6 * radius, 3)
                if np.linalg.norm(c) <= 0.6 * radius:
                    break
            ax = rng.uniform(0.05, 0.45, 3) * radius
            rot = random_rotation(rng)
            big = float(ax.max())
        val = rng.random()
        if np.linalg.norm(c) + big <= 0.95 * radius:
            C.append(c)
            AX.append(ax)
            ROT.append(rot)
            VAL.append(val)
    return dict(dim=dim, centres=np.array(C), axes=np.array(AX), rot=np.array(ROT),
                values=np.array(VAL), scale=1.0)


def scaled(ph: dict, s: float) -> dict:
    out = dict(ph)
    out["values"] = ph["values"] * s
    out["scale"] = ph.get("scale", 1.0) * s
    return out


# ---------------------------------------------------------------------------
# the scanner's measurement lines (independent of the oracle and the library)
# ---------------------------------------------------------------------------
def rays_of(spec: dict, view_ids=None, xp=np, device=None):
    """Measurement lines of a geometry spec as (origin, unit direction), FP64.

    Returns arrays of shape (n_views_selected * nv * nu, 3) in [view][v][u] order.
    """
    kind = spec["kind"]
    nu, nv = spec["nu"], spec.get("nv", 1)
    if kind == "custom3d":
        poses = np.asarray(spec["poses"], np.float64).reshape(-1, 12)
        V = poses.shape[0]
    else:
        ang = np.asarray(spec["angles"], np.float64)
        V = ang.shape[0]
    views = np.arange(V) if view_ids is None else np.asarray(view_ids, np.int64)

    def arr(a):
        a = np.asarray(a, np.float64)
        if xp is np:
            return a
        return xp.as_tensor(a, dtype=xp.float64, device=device)

    uu = arr((np.arange(nu) - 0.5 * (nu - 1)) * spec["pu"])
    vv = arr((np.arange(nv) - 0.5 * (nv - 1)) * spec.get("pv", 1.0))
    if kind == "custom3d":
        p = poses[views]
        S, Cc, eu, ev = p[:, 0:3], p[:, 3:6], p[:, 6:9], p[:, 9:12]
    else:
        t = ang[views]
        c, s = np.cos(t), np.sin(t)
        z = np.zeros_like(t)
        dc = np.stack([-c, -s, z], 1)
        eu = np.stack([-s, c, z], 1)
        ev = np.stack([z, z, np.ones_like(t)], 1)
        S = spec.get("sod", 0.0) * np.stack([c, s, z], 1)
        Cc = S + spec.get("sdd", 0.0) * dc
    S, Cc, eu, ev = arr(S), arr(Cc), arr(eu), arr(ev)
    nV = S.shape[0]
    # broadcast to (views, nv, nu, 3)
    U = uu.reshape(1, 1, nu, 1)
    W = vv.reshape(1, nv, 1, 1)
    eu_ = eu.reshape(nV, 1, 1, 3)
    ev_ = ev.reshape(nV, 1, 1, 3)
    if kind == "parallel2d":
        t = ang[views]
        dc_ = arr(np.stack([-np.cos(t), -np.sin(t), np.zeros_like(t)], 1)).reshape(nV, 1, 1, 3)
        org = U * eu_ + 0.0 * W
        d = dc_ + 0.0 * U + 0.0 * W
    elif kind == "fan2d_curved":
        t = ang[views]
        dc_ = arr(np.stack([-np.cos(t), -np.sin(t), np.zeros_like(t)], 1)).reshape(nV, 1, 1, 3)
        org = S.reshape(nV, 1, 1, 3) + 0.0 * U + 0.0 * W
        d = xp.cos(U) * dc_ + xp.sin(U) * eu_ + 0.0 * W
    else:
        P = Cc.reshape(nV, 1, 1, 3) + U * eu_ + W * ev_
        org = S.reshape(nV, 1, 1, 3) + 0.0 * P
        d = P - S.reshape(nV, 1, 1, 3)
    org = org.reshape(-1, 3)
    d = d.reshape(-1, 3)
    if xp is np:
        d = d / np.linalg.norm(d, axis=1, keepdims=True)
    else:
        d = d / xp.linalg.norm(d, dim=1, keepdim=True)
    return org, d


def line_integrals(ph: dict, org, d, xp=np):
    """Exact sum over shapes of value * chord length of each line (unit d), FP64."""
    dim = ph["dim"]
    out = xp.zeros(org.shape[0], dtype=org.dtype, **({} if xp is np else {"device": org.device}))
    for k in range(ph["centres"].shape[0]):
        c = ph["centres"][k]
        ax = ph["axes"][k].copy()
        R = ph["rot"][k]
        if dim == 2:
            ax[2] = 1.0
        Rt = R.T
        if xp is not np:
            c = xp.as_tensor(c, dtype=org.dtype, device=org.device)
            Rt = xp.as_tensor(Rt, dtype=org.dtype, device=org.device)
            inv = xp.as_tensor(1.0 / ax, dtype=org.dtype, device=org.device)
        else:
            inv = 1.0 / ax
        o2 = ((org - c) @ Rt.T) * inv
        d2 = (d @ Rt.T) * inv
        if dim == 2:
            o2 = o2[:, :2]
            d2 = d2[:, :2]
        a = (d2 * d2).sum(1)
        b = 2.0 * (o2 * d2).sum(1)
        cc = (o2 * o2).sum(1) - 1.0
        disc = b * b - 4.0 * a * cc
        pos = disc > 0
        if xp is np:
            root = np.sqrt(np.where(pos, disc, 0.0))
        else:
            root = xp.sqrt(xp.where(pos, disc, xp.zeros_like(disc)))
        out = out + float(ph["values"][k]) * root / a
    return out


def pixelize(ph: dict, n, h: float, sub: int = 4, xp=np, device=None):
    """Voxel averages of the phantom by sub^dim point samples per voxel (FP64).

    Returns a flat array in x-fastest order.
    """
    dim = ph["dim"]
    n = tuple(int(v) for v in n)
    offs = (np.arange(sub) + 0.5) / sub
    lo = [-0.5 * n[a] * h for a in range(dim)]
    def coords(a):
        c = lo[a] + (np.arange(n[a])[:, None] + offs[None, :]) * h
        return c.reshape(-1)
    if xp is np:
        mk = lambda a: a
    else:
        mk = lambda a: xp.as_tensor(a, dtype=xp.float64, device=device)
    if dim == 2:
        xs, ys = mk(coords(0)), mk(coords(1))
        acc = xp.zeros((n[1] * sub, n[0] * sub), dtype=xs.dtype, **({} if xp is np else {"device": device}))
        Y = ys[:, None]
        X = xs[None, :]
        for k in range(ph["centres"].shape[0]):
            c = ph["centres"][k]; ax = ph["axes"][k]; R = ph["rot"][k]
            dx, dy = X - c[0], Y - c[1]
            u = (R[0, 0] * dx + R[1, 0] * dy) / ax[0]
            v = (R[0, 1] * dx + R[1, 1] * dy) / ax[1]
            acc = acc + float(ph["values"][k]) * ((u * u + v * v) <= 1.0)
        acc = acc.reshape(n[1], sub, n[0], sub).mean(axis=(1, 3)) if xp is np else \
            acc.reshape(n[1], sub, n[0], sub).mean(dim=(1, 3))
        return acc.reshape(-1)
    # 3D: slab by slab in z to bound memory
    out = []
    xs, ys = mk(coords(0)), mk(coords(1))
    zc = coords(2)
    for iz in range(n[2]):
        zs = mk(zc[iz * sub:(iz + 1) * sub])
        Z = zs[:, None, None]
        Y = ys[None, :, None]
        X = xs[None, None, :]
        acc = 0.0
        for k in range(ph["centres"].shape[0]):
            c = ph["centres"][k]; ax = ph["axes"][k]; R = ph["rot"][k]
            dx, dy, dz = X - c[0], Y - c[1], Z - c[2]
            u = (R[0, 0] * dx + R[1, 0] * dy + R[2, 0] * dz) / ax[0]
            v = (R[0, 1] * dx + R[1, 1] * dy + R[2, 1] * dz) / ax[1]
            w = (R[0, 2] * dx + R[1, 2] * dy + R[2, 2] * dz) / ax[2]
            acc = acc + float(ph["values"][k]) * ((u * u + v * v + w * w) <= 1.0)
        if xp is np:
            sl = acc.reshape(sub, n[1], sub, n[0], sub).mean(axis=(0, 2, 4))
        else:
            sl = acc.reshape(sub, n[1], sub, n[0], sub).mean(dim=(0, 2, 4))
        out.append(sl.reshape(-1))
    return np.concatenate(out) if xp is np else xp.cat(out)


# ---------------------------------------------------------------------------
# noise
# ---------------------------------------------------------------------------
def add_gaussian(y: np.ndarray, rel_sigma: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma = rel_sigma * float(np.max(y))
    return y + sigma * rng.standard_normal(y.shape[0])


def add_poisson(y: np.ndarray, n0: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.poisson(n0 * np.exp(-y))
    return np.log(n0 / np.maximum(k, 1))
