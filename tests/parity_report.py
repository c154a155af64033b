"""Error statistics of a GPU-vs-oracle comparison against the plain bound.

The plain bound on a ray sum (or a voxel sum) is

    |gpu - oracle| <= 1e-5 * max(|ref|, 1e-3 * max|ref|),

a 1e-5 relative error with a floor at 1e-3 of the largest reference value for
sums near zero.  The GPU places every line in FP32 to about 1e-5 voxel, so a
line that only grazes a tile or a voxel has a length with a larger relative
error than that; the parity tests therefore assert the derived tolerance of
``test_gpu_parity.py`` on every element and, beside it, how many elements
exceed the plain bound (``frac_over``) and by how much (``max_ratio``).

``record`` returns those statistics; when the environment variable
CSGD_PARITY_REPORT names a file, it also appends them to it as one JSON line.
"""
from __future__ import annotations

import json
import os

import numpy as np


def plain_bound(ref) -> np.ndarray:
    a = np.abs(np.asarray(ref, np.float64))
    top = float(a.max()) if a.size else 0.0
    return 1e-5 * np.maximum(a, 1e-3 * top)


def record(case: str, kind: str, got, ref, **extra) -> dict:
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    bound = plain_bound(ref)
    over = err > bound
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(bound > 0, err / bound, np.where(err > 0, np.inf, 0.0))
    st = dict(case=case, kind=kind, n=int(err.size), n_over=int(over.sum()),
              frac_over=float(over.mean()) if err.size else 0.0,
              max_ratio=float(ratio.max()) if err.size else 0.0,
              max_abs_err=float(err.max()) if err.size else 0.0,
              max_abs_ref=float(np.abs(ref).max()) if ref.size else 0.0)
    st.update(extra)
    path = os.environ.get("CSGD_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(st) + "\n")
    return st
