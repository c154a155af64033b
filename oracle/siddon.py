"""ctypes front end of ``siddon.c`` (the FP64 alpha-merge Siddon of Sec. II-A).

Test infrastructure only (see the package docstring).  The shared object is
compiled with gcc on first use when it is missing or older than its source;
``__graft_entry__.build()`` also compiles it.

Pinned by ``tests/test_oracle_siddon.py``: brute-force slab clipping of every
(ray, voxel) pair, axis-aligned and 45-degree closed forms, the bounding-box
chord, and analytic ellipse/ellipsoid line integrals.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon.c")
_SO = os.path.join(_HERE, "_siddon_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``siddon.c`` into ``_siddon_oracle.so`` (gcc, OpenMP, FP64)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64p = ctypes.POINTER(ctypes.c_int64)
            f64p = ctypes.POINTER(ctypes.c_double)
            common = [ctypes.c_int, i64p, ctypes.c_double, f64p, ctypes.c_int64, f64p, f64p]
            lib.oracle_siddon_count.argtypes = common + [i64p]
            lib.oracle_siddon_count.restype = ctypes.c_int64
            lib.oracle_siddon_fill.argtypes = common + [i64p, i64p, f64p]
            lib.oracle_siddon_fill.restype = None
            lib.oracle_project_box.argtypes = common + [i64p, i64p, f64p, f64p]
            lib.oracle_project_box.restype = None
            lib.oracle_backproject_box.argtypes = common + [i64p, i64p, f64p, f64p]
            lib.oracle_backproject_box.restype = None
            lib.oracle_count_box.argtypes = common + [i64p, i64p]
            lib.oracle_count_box.restype = ctypes.c_int64
            lib.oracle_num_threads.restype = ctypes.c_int
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _grid_args(grid):
    dim = len(grid.n)
    n = np.ones(3, np.int64)
    n[:dim] = grid.n
    lo = np.zeros(3, np.float64)
    lo[:dim] = grid.lo
    return dim, n, float(grid.h), lo


def _rays(org, dirs):
    org = np.ascontiguousarray(org, np.float64).reshape(-1, 3)
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    assert org.shape == dirs.shape
    return org, dirs


def system_matrix(grid, org, dirs) -> sp.csr_matrix:
    """Rows of A for the given rays as a CSR matrix (n_rays x n_voxels), FP64.

    Entry (i, j) is the intersection length of line i with voxel j (Sec. II-A).
    """
    lib = _load()
    dim, n, h, lo = _grid_args(grid)
    org, dirs = _rays(org, dirs)
    nr = org.shape[0]
    counts = np.zeros(nr, np.int64)
    i64 = ctypes.c_int64
    f64 = ctypes.c_double
    total = lib.oracle_siddon_count(dim, _p(n, i64), h, _p(lo, f64), nr, _p(org, f64),
                                    _p(dirs, f64), _p(counts, i64))
    offsets = np.zeros(nr + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    cols = np.zeros(max(total, 1), np.int64)
    vals = np.zeros(max(total, 1), np.float64)
    lib.oracle_siddon_fill(dim, _p(n, i64), h, _p(lo, f64), nr, _p(org, f64), _p(dirs, f64),
                           _p(offsets, i64), _p(cols, i64), _p(vals, f64))
    nvox = int(np.prod(grid.n))
    return sp.csr_matrix((vals[:total], cols[:total], offsets), shape=(nr, nvox))


def project_box(grid, org, dirs, box_lo, box_hi, x) -> np.ndarray:
    """out_i = sum over voxels j inside the index box of A_ij x_j (FP64)."""
    lib = _load()
    dim, n, h, lo = _grid_args(grid)
    org, dirs = _rays(org, dirs)
    blo = np.zeros(3, np.int64)
    bhi = np.ones(3, np.int64)
    blo[:dim] = box_lo
    bhi[:dim] = box_hi
    x = np.ascontiguousarray(x, np.float64).reshape(-1)
    out = np.zeros(org.shape[0], np.float64)
    i64 = ctypes.c_int64
    f64 = ctypes.c_double
    lib.oracle_project_box(dim, _p(n, i64), h, _p(lo, f64), org.shape[0], _p(org, f64),
                           _p(dirs, f64), _p(blo, i64), _p(bhi, i64), _p(x, f64), _p(out, f64))
    return out


def backproject_box(grid, org, dirs, box_lo, box_hi, r) -> np.ndarray:
    """g_j = sum_i A_ij r_i for voxels j inside the index box, 0 elsewhere (FP64)."""
    lib = _load()
    dim, n, h, lo = _grid_args(grid)
    org, dirs = _rays(org, dirs)
    blo = np.zeros(3, np.int64)
    bhi = np.ones(3, np.int64)
    blo[:dim] = box_lo
    bhi[:dim] = box_hi
    r = np.ascontiguousarray(r, np.float64).reshape(-1)
    assert r.shape[0] == org.shape[0]
    g = np.zeros(int(np.prod(grid.n)), np.float64)
    i64 = ctypes.c_int64
    f64 = ctypes.c_double
    lib.oracle_backproject_box(dim, _p(n, i64), h, _p(lo, f64), org.shape[0], _p(org, f64),
                               _p(dirs, f64), _p(blo, i64), _p(bhi, i64), _p(r, f64), _p(g, f64))
    return g


def count_box(grid, org, dirs, box_lo, box_hi) -> int:
    """Number of non-zeros A_ij with voxel j inside the index box."""
    lib = _load()
    dim, n, h, lo = _grid_args(grid)
    org, dirs = _rays(org, dirs)
    blo = np.zeros(3, np.int64)
    bhi = np.ones(3, np.int64)
    blo[:dim] = box_lo
    bhi[:dim] = box_hi
    i64 = ctypes.c_int64
    f64 = ctypes.c_double
    return int(lib.oracle_count_box(dim, _p(n, i64), h, _p(lo, f64), org.shape[0], _p(org, f64),
                                    _p(dirs, f64), _p(blo, i64), _p(bhi, i64)))
