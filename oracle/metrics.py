"""Quality measures of Sec. III (oracle, FP64).

Test infrastructure only (see the package docstring).

SNR = 20 log10(||x_true|| / ||x_true - x_est||) and observation gap =
20 log10(||y|| / ||y - A x_est||), both as defined at the start of Sec. III; the
observation gap uses the true residual y - A x (a full forward projection), not
the solver's running residual.  RMSE = sqrt(mean((x - x_ref)^2)) is the
measure the parity tests use.

Parity: closed-form values on hand-made vectors in ``tests/test_oracle_solver.py``.
"""
from __future__ import annotations

import numpy as np

from . import siddon
from .geometry import Geometry


def snr_db(x_true, x_est) -> float:
    x_true = np.asarray(x_true, np.float64).ravel()
    e = x_true - np.asarray(x_est, np.float64).ravel()
    return float(20.0 * np.log10(np.linalg.norm(x_true) / np.linalg.norm(e)))


def forward_full(geom: Geometry, x) -> np.ndarray:
    """A x over all rays and all voxels."""
    org, d = geom.rays()
    n = geom.n
    return siddon.project_box(geom.grid, org, d, [0] * len(n), list(n), x)


def observation_gap_db(geom: Geometry, y, x_est) -> float:
    y = np.asarray(y, np.float64).ravel()
    res = y - forward_full(geom, x_est)
    return float(20.0 * np.log10(np.linalg.norm(y) / np.linalg.norm(res)))


def rmse(a, b) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.sqrt(np.mean((a - b) ** 2)))
