"""Seeded measurement data for a workload: y = exact line integrals + noise.

``make_data(cfg)`` returns (y, phantom) where y is an FP32 numpy array in
[view][v][u] order and phantom the (possibly rescaled) shape parameters; with
``device='cuda'`` the line integrals are evaluated with torch on the GPU (FP64)
for the large workloads, the noise always with numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

from . import phantom as PH


def make_data(cfg: dict, device: str | None = None, chunk_views: int = 8):
    geom = cfg["geom"]
    dim = len(geom["n"])
    radius = 0.5 * geom["n"][0] * geom.get("h", 1.0)
    ph = PH.make_phantom(dim, cfg["phantom"]["n_shapes"], radius, cfg["phantom"]["seed"])
    n_views = len(geom["angles"]) if geom["kind"] != "custom3d" else len(geom["poses"])
    parts = []
    if device is None:
        for v0 in range(0, n_views, chunk_views):
            views = np.arange(v0, min(n_views, v0 + chunk_views))
            o, d = PH.rays_of(geom, views)
            parts.append(PH.line_integrals(ph, o, d))
        y = np.concatenate(parts)
    else:
        import torch
        for v0 in range(0, n_views, chunk_views):
            views = np.arange(v0, min(n_views, v0 + chunk_views))
            o, d = PH.rays_of(geom, views, xp=torch, device=device)
            parts.append(PH.line_integrals(ph, o, d, xp=torch).cpu().numpy())
        y = np.concatenate(parts)
    noise = cfg["noise"]
    if noise["kind"] == "gaussian":
        y = PH.add_gaussian(y, noise["level"], noise["seed"])
    elif noise["kind"] == "poisson":
        s = 4.0 / float(np.max(y))
        ph = PH.scaled(ph, s)
        y = PH.add_poisson(y * s, noise["level"], noise["seed"])
    return y.astype(np.float32), ph
