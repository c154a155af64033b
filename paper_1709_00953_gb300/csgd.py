"""Python binding of the C ABI in include/csgd.h (argument marshalling only).

Every computation happens in ``libcsgd.so`` (CUDA, sm_103a).  This module only
converts Python values and torch tensors into the ABI's plain pointers and
sizes, and turns non-zero status codes into ``CsgdError``.  There is no CPU
fallback: if the library is missing, every call raises.

Function names follow the ABI: ``geometry_create``, ``block_partition``,
``project_block``, ``backproject_block``, ``solve_step``, ``solve`` ...
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcsgd.so")

KINDS = {"parallel2d": 0, "fan2d_flat": 1, "fan2d_curved": 2, "cone3d": 3, "custom3d": 4}
SEQUENTIAL, UNIFORM, IMPORTANCE, MIXED = 0, 1, 2, 3
SYNC_COLUMN, SYNC_EPOCH = 0, 1
SCATTER = -1  # bp_groups value of the ray-driven scatter backprojection
BRICK = -2    # bp_groups values -2, -3, -4: the brick backprojection (no ray table)
BRICKS = (-2, -3, -4)  # with brick shapes 0, 1, 2 (3D 16x16x{16,8,4}, 2D {32,16,8}^2)


class CsgdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("csgd error %d: %s" % (code, msg))
        self.code = code


# ---------------------------------------------------------------------------
# ABI structs
# ---------------------------------------------------------------------------
class GeometryDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("h", ctypes.c_double),
                ("n_views", ctypes.c_int32), ("angles", ctypes.POINTER(ctypes.c_double)),
                ("poses", ctypes.POINTER(ctypes.c_double)), ("nu", ctypes.c_int32),
                ("nv", ctypes.c_int32), ("pu", ctypes.c_double), ("pv", ctypes.c_double),
                ("sod", ctypes.c_double), ("sdd", ctypes.c_double)]


class PartitionDesc(ctypes.Structure):
    _fields_ = [("tiles", ctypes.c_int32 * 3), ("view_blocks", ctypes.c_int32),
                ("view_block_of", ctypes.POINTER(ctypes.c_int32)),
                ("det_blocks_u", ctypes.c_int32), ("det_blocks_v", ctypes.c_int32)]


class PartitionInfo(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("n_rays", ctypes.c_int64),
                ("n_voxels", ctypes.c_int64), ("z_floats", ctypes.c_int64)]


class SolverParams(ctypes.Structure):
    _fields_ = [("sampling", ctypes.c_int32), ("sync", ctypes.c_int32),
                ("group_size", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("gamma", ctypes.c_double), ("b", ctypes.c_double),
                ("theta_step", ctypes.c_double), ("seed", ctypes.c_uint64)]


class BlockChoice(ctypes.Structure):
    _fields_ = [("j", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("row_blocks", ctypes.POINTER(ctypes.c_int32))]


class StepInfo(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("j", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("beta", ctypes.c_double), ("gg", ctypes.c_double), ("qq", ctypes.c_double),
                ("mu", ctypes.c_double), ("nnz", ctypes.c_int64)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 4), ("ms", ctypes.c_double * 4)]


KERNEL_KINDS = ("backproject", "forward_dual", "epilogue", "epoch_close")


class Report(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("epochs", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("updates", ctypes.c_double), ("residual_norm", ctypes.c_double),
                ("rays", ctypes.c_int64), ("tile_voxels", ctypes.c_int64)]


class BatchParams(ctypes.Structure):
    _fields_ = [("wait_limit_ns", ctypes.c_int64), ("stall_last_task", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


# every symbol include/csgd.h declares, with its signature
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
SIGNATURES = {
    "csgd_geometry_create": ([ctypes.POINTER(GeometryDesc), ctypes.POINTER(_vp)], _i32),
    "csgd_geometry_destroy": ([_vp], _i32),
    "csgd_block_partition": ([_vp, ctypes.POINTER(PartitionDesc), ctypes.POINTER(_vp)], _i32),
    "csgd_partition_destroy": ([_vp], _i32),
    "csgd_partition_get_info": ([_vp, ctypes.POINTER(PartitionInfo)], _i32),
    "csgd_partition_probabilities": ([_vp, ctypes.POINTER(ctypes.c_double)], _i32),
    "csgd_project_block": ([_vp, ctypes.POINTER(_i32), _i32, _i32, _vp, _vp, _i32, _vp], _i32),
    "csgd_backproject_block": ([_vp, ctypes.POINTER(_i32), _i32, _i32, _vp, _vp, _i32, _vp], _i32),
    "csgd_project_full": ([_vp, _vp, _vp, _vp], _i32),
    "csgd_backproject_block_noalloc": ([_vp, ctypes.POINTER(_i32), _i32, _i32, _vp, _vp, _i32, _vp],
                                       _i32),
    "csgd_schedule_generate": ([_vp, ctypes.POINTER(SolverParams), _i32, ctypes.POINTER(_i32),
                                _i64, ctypes.POINTER(_i64)], _i32),
    "csgd_solver_footprint_bytes": ([_vp, ctypes.POINTER(SolverParams), ctypes.POINTER(_i64)], _i32),
    "csgd_solver_create": ([_vp, ctypes.POINTER(SolverParams), _vp, _vp, ctypes.POINTER(_vp)], _i32),
    "csgd_solver_destroy": ([_vp], _i32),
    "csgd_solver_reset": ([_vp, _vp, _i32, _vp], _i32),
    "csgd_solve_step": ([_vp, ctypes.POINTER(BlockChoice), ctypes.POINTER(StepInfo), _vp], _i32),
    "csgd_solve": ([_vp, _i64, _vp, _i32, ctypes.POINTER(Report), _i32, _vp], _i32),
    "csgd_solver_history": ([_vp, ctypes.POINTER(StepInfo), _i64, ctypes.POINTER(_i64)], _i32),
    "csgd_solver_state_bytes": ([_vp, ctypes.POINTER(_i64)], _i32),
    "csgd_solver_set_launch": ([_vp, _i32, _i32], _i32),
    "csgd_solver_autotune": ([_vp, _i64, ctypes.POINTER(_i32), ctypes.POINTER(_i32), _vp], _i32),
    "csgd_solver_get_state": ([_vp, _vp, _i64, _vp], _i32),
    "csgd_solver_set_state": ([_vp, _vp, _i64, _vp], _i32),
    "csgd_solver_graph_create": ([_vp, _i64, _vp, _i32, ctypes.POINTER(_vp)], _i32),
    "csgd_graph_batch_create": ([ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp)], _i32),
    "csgd_graph_launch": ([_vp, _vp], _i32),
    "csgd_graph_destroy": ([_vp], _i32),
    "csgd_batch_create": ([ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_vp), _i32,
                           ctypes.POINTER(BatchParams), ctypes.POINTER(_vp)], _i32),
    "csgd_batch_launch": ([_vp, _vp], _i32),
    "csgd_batch_status": ([_vp], _i32),
    "csgd_batch_info": ([_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i64), ctypes.POINTER(_i32)], _i32),
    "csgd_batch_destroy": ([_vp], _i32),
    "csgd_solver_profile": ([_vp, _i32], _i32),
    "csgd_solver_profile_read": ([_vp, ctypes.POINTER(KernelTimes), _i32], _i32),
    "csgd_last_error": ([], ctypes.c_char_p),
    "csgd_version": ([], ctypes.c_char_p),
}

_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libcsgd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise CsgdError(-6, "libcsgd.so not built (run __graft_entry__.build()): %s" % p)
            lib = ctypes.CDLL(p)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise CsgdError(rc, load().csgd_last_error().decode())


def _stream(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, name, n=None):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float32 CUDA tensor" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t, name, n):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float32 CPU tensor" % name)
    if t.numel() != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), n))
    return ctypes.c_void_p(t.data_ptr())


def version() -> str:
    return load().csgd_version().decode()


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
class Geometry:
    def __init__(self, spec: dict):
        lib = load()
        self.spec = dict(spec)
        kind = KINDS[spec["kind"]]
        n = list(spec["n"]) + [1] * (3 - len(spec["n"]))
        d = GeometryDesc()
        d.kind = kind
        for a in range(3):
            d.n[a] = int(n[a])
        d.h = float(spec.get("h", 1.0))
        self._angles = None
        self._poses = None
        if kind == 4:
            self._poses = np.ascontiguousarray(spec["poses"], np.float64).reshape(-1)
            d.n_views = self._poses.shape[0] // 12
            d.poses = self._poses.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        else:
            self._angles = np.ascontiguousarray(spec["angles"], np.float64).reshape(-1)
            d.n_views = self._angles.shape[0]
            d.angles = self._angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.nu = int(spec["nu"])
        d.nv = int(spec.get("nv", 1))
        d.pu = float(spec["pu"])
        d.pv = float(spec.get("pv", 1.0))
        d.sod = float(spec.get("sod", 0.0))
        d.sdd = float(spec.get("sdd", 0.0))
        h = ctypes.c_void_p()
        _check(lib.csgd_geometry_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.n_views = d.n_views
        self.n_rays = d.n_views * d.nu * (d.nv if kind >= 3 else 1)
        self.n_voxels = int(np.prod(n))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.csgd_geometry_destroy(self.handle)
            self.handle = None


def geometry_create(spec: dict) -> Geometry:
    return Geometry(spec)


class Partition:
    def __init__(self, geom: Geometry, tiles, view_blocks=1, det_blocks=(1, 1), view_block_of=None):
        lib = load()
        self.geom = geom
        d = PartitionDesc()
        t = list(tiles) + [1] * (3 - len(tiles))
        for a in range(3):
            d.tiles[a] = int(t[a])
        d.view_blocks = int(view_blocks)
        self._vbo = None
        if view_block_of is not None:
            self._vbo = np.ascontiguousarray(view_block_of, np.int32)
            d.view_block_of = self._vbo.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        db = tuple(det_blocks) + (1,)
        d.det_blocks_u = int(db[0])
        d.det_blocks_v = int(db[1])
        h = ctypes.c_void_p()
        _check(lib.csgd_block_partition(geom.handle, ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        info = PartitionInfo()
        _check(lib.csgd_partition_get_info(h, ctypes.byref(info)))
        self.m, self.n = info.m, info.n
        self.n_rays, self.n_voxels, self.z_floats = info.n_rays, info.n_voxels, info.z_floats

    def probabilities(self) -> np.ndarray:
        P = np.zeros((self.m, self.n), np.float64)
        _check(load().csgd_partition_probabilities(self.handle,
                                                   P.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return P

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.csgd_partition_destroy(self.handle)
            self.handle = None


def block_partition(geom: Geometry, tiles, view_blocks=1, det_blocks=(1, 1),
                    view_block_of=None) -> Partition:
    return Partition(geom, tiles, view_blocks, det_blocks, view_block_of)


def _rows(row_blocks):
    arr = np.ascontiguousarray(np.asarray(row_blocks, np.int32).reshape(-1))
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def project_block(part: Partition, row_blocks, j: int, x, out, accumulate=False, stream=None):
    """out[rows of I] = (+=) A_I^J x_J   (x: volume, out: sinogram; CUDA float32)."""
    arr, ptr = _rows(row_blocks)
    _check(load().csgd_project_block(part.handle, ptr, arr.shape[0], int(j),
                                     _dev_ptr(x, "x", part.n_voxels),
                                     _dev_ptr(out, "out", part.n_rays), int(bool(accumulate)),
                                     _stream(stream)))


def backproject_block(part: Partition, row_blocks, j: int, r, g, accumulate=False, stream=None):
    """g[voxels of J] = (+=) (A_I^J)^T r_I   (r: sinogram, g: volume; CUDA float32)."""
    arr, ptr = _rows(row_blocks)
    _check(load().csgd_backproject_block(part.handle, ptr, arr.shape[0], int(j),
                                         _dev_ptr(r, "r", part.n_rays),
                                         _dev_ptr(g, "g", part.n_voxels), int(bool(accumulate)),
                                         _stream(stream)))


NOALLOC_MAX_RAYS = 262144  # CSGD_NOALLOC_MAX_RAYS of include/csgd.h


def backproject_block_noalloc(part: Partition, row_blocks, j: int, r, g, accumulate=False,
                              stream=None):
    """Same as backproject_block, for callers that cannot allocate device memory.

    The library keeps this call's scratch in a fixed 8 MiB array on the GPU
    instead of allocating it, so it works where cudaMalloc is not allowed (after
    start-up in a real-time loop, or when all device memory is handed out in
    advance).  At most NOALLOC_MAX_RAYS rays per call; one ordinary device call
    with the partition must come first (it uploads the partition's tables);
    concurrent calls share the array and must not overlap on the GPU.
    """
    arr, ptr = _rows(row_blocks)
    _check(load().csgd_backproject_block_noalloc(part.handle, ptr, arr.shape[0], int(j),
                                                 _dev_ptr(r, "r", part.n_rays),
                                                 _dev_ptr(g, "g", part.n_voxels),
                                                 int(bool(accumulate)), _stream(stream)))


def project_full(part: Partition, x, out, stream=None):
    _check(load().csgd_project_full(part.handle, _dev_ptr(x, "x", part.n_voxels),
                                    _dev_ptr(out, "out", part.n_rays), _stream(stream)))


def solver_params(sampling=IMPORTANCE, alpha=1.0, gamma=1.0, b=1.0, group_size=1, sync=SYNC_COLUMN,
                  seed=0, theta_step=1.0 / 40.0) -> SolverParams:
    p = SolverParams()
    p.sampling = int(sampling)
    p.sync = int(sync)
    p.group_size = int(group_size)
    p.alpha = float(alpha)
    p.gamma = float(gamma)
    p.b = float(b)
    p.theta_step = float(theta_step)
    p.seed = int(seed) & ((1 << 64) - 1)
    return p


def schedule_generate(part: Partition, params: dict, n_epochs: int) -> list:
    prm = solver_params(**params)
    n = ctypes.c_int64(0)
    load().csgd_schedule_generate(part.handle, ctypes.byref(prm), int(n_epochs), None, 0,
                                  ctypes.byref(n))
    buf = np.zeros(max(1, n.value), np.int32)
    _check(load().csgd_schedule_generate(part.handle, ctypes.byref(prm), int(n_epochs),
                                         buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         buf.shape[0], ctypes.byref(n)))
    return buf[:n.value].tolist()


def footprint_bytes(part: Partition, params: dict) -> int:
    prm = solver_params(**params)
    n = ctypes.c_int64(0)
    _check(load().csgd_solver_footprint_bytes(part.handle, ctypes.byref(prm), ctypes.byref(n)))
    return n.value


class Solver:
    def __init__(self, part: Partition, params: dict, y, stream=None):
        self.part = part
        self.params = dict(params)
        prm = solver_params(**params)
        h = ctypes.c_void_p()
        _check(load().csgd_solver_create(part.handle, ctypes.byref(prm),
                                         _dev_ptr(y, "y", part.n_rays), _stream(stream),
                                         ctypes.byref(h)))
        self.handle = h

    def reset(self, y, stream=None):
        if y.is_cuda:
            ptr, host = _dev_ptr(y, "y", self.part.n_rays), 0
        else:
            ptr, host = _host_ptr(y, "y", self.part.n_rays), 1
        _check(load().csgd_solver_reset(self.handle, ptr, host, _stream(stream)))

    def step(self, j=None, row_blocks=None, stream=None) -> dict:
        info = StepInfo()
        if j is None:
            _check(load().csgd_solve_step(self.handle, None, ctypes.byref(info), _stream(stream)))
        else:
            arr, ptr = _rows(row_blocks)
            ch = BlockChoice(int(j), arr.shape[0], ptr)
            _check(load().csgd_solve_step(self.handle, ctypes.byref(ch), ctypes.byref(info),
                                          _stream(stream)))
        return dict(step=info.step, j=info.j, n_rows=info.n_rows, beta=info.beta, gg=info.gg,
                    qq=info.qq, mu=info.mu)

    def solve(self, n_steps: int, x_out=None, report=True, residual=False, stream=None):
        rep = Report()
        if x_out is None:
            ptr, host = None, 0
        elif x_out.is_cuda:
            ptr, host = _dev_ptr(x_out, "x_out", self.part.n_voxels), 0
        else:
            ptr, host = _host_ptr(x_out, "x_out", self.part.n_voxels), 1
        _check(load().csgd_solve(self.handle, int(n_steps), ptr, host,
                                 ctypes.byref(rep) if report else None, int(bool(residual)),
                                 _stream(stream)))
        if not report:
            return None
        return dict(steps=rep.steps, epochs=rep.epochs, nnz=rep.nnz, updates=rep.updates,
                    residual_norm=rep.residual_norm, rays=rep.rays, tile_voxels=rep.tile_voxels)

    def history(self, capacity: int = 1 << 20) -> list:
        cnt = ctypes.c_int64(0)
        buf = (StepInfo * max(1, capacity))()
        _check(load().csgd_solver_history(self.handle, buf, capacity, ctypes.byref(cnt)))
        return [dict(step=buf[k].step, beta=buf[k].beta, gg=buf[k].gg, qq=buf[k].qq, mu=buf[k].mu,
                     nnz=buf[k].nnz) for k in range(cnt.value)]

    def graph(self, n_steps: int, x_out=None) -> "Graph":
        """A CUDA graph of a whole solve (reset, n_steps steps, x to x_out)."""
        if x_out is None:
            ptr, host = None, 0
        elif x_out.is_cuda:
            ptr, host = _dev_ptr(x_out, "x_out", self.part.n_voxels), 0
        else:
            ptr, host = _host_ptr(x_out, "x_out", self.part.n_voxels), 1
        h = ctypes.c_void_p()
        _check(load().csgd_solver_graph_create(self.handle, int(n_steps), ptr, host, ctypes.byref(h)))
        return Graph(h, [self, x_out])

    def set_launch(self, bp_groups: int = 0, fwd_lanes: int = 0):
        """Launch shapes of the kernels (0 = the library's models): view groups
        per gather CTA 1..8, SCATTER (-1) for the ray-driven backprojection with
        global atomics, or BRICK (-2) for the brick backprojection; lanes per
        ray 1, 2 or 4."""
        _check(load().csgd_solver_set_launch(self.handle, int(bp_groups), int(fwd_lanes)))

    def autotune(self, trial_steps: int, stream=None) -> tuple:
        """Times every launch shape over the first trial_steps steps, keeps the
        fastest and resets the solver; returns (bp_groups, fwd_lanes), with
        bp_groups = SCATTER (-1) or BRICK (-2) if one of those backprojections won."""
        c, l = ctypes.c_int32(), ctypes.c_int32()
        _check(load().csgd_solver_autotune(self.handle, int(trial_steps), ctypes.byref(c),
                                           ctypes.byref(l), _stream(stream)))
        return c.value, l.value

    def state(self, stream=None) -> np.ndarray:
        """Checkpoint: the solver's whole iteration state as a host byte array."""
        n = ctypes.c_int64()
        _check(load().csgd_solver_state_bytes(self.handle, ctypes.byref(n)))
        buf = np.zeros(int(n.value), dtype=np.uint8)
        _check(load().csgd_solver_get_state(self.handle, buf.ctypes.data, buf.size, _stream(stream)))
        return buf

    def set_state(self, buf, stream=None):
        """Resume from a checkpoint taken by state() (same partition and parameters)."""
        arr = np.ascontiguousarray(np.asarray(buf, dtype=np.uint8))
        _check(load().csgd_solver_set_state(self.handle, arr.ctypes.data, arr.size, _stream(stream)))

    def profile(self, enable: bool = True):
        _check(load().csgd_solver_profile(self.handle, int(bool(enable))))

    def profile_read(self, reset: bool = True) -> dict:
        t = KernelTimes()
        _check(load().csgd_solver_profile_read(self.handle, ctypes.byref(t), int(bool(reset))))
        return {KERNEL_KINDS[k]: dict(launches=t.launches[k], ms=t.ms[k]) for k in range(4)}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.csgd_solver_destroy(self.handle)
            self.handle = None


class Graph:
    """A captured solve (or a batch of them); keeps its solvers and outputs alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(load().csgd_graph_launch(self.handle, _stream(stream)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.csgd_graph_destroy(self.handle)
            self.handle = None


def graph_batch(graphs) -> Graph:
    """One graph running the given solve graphs concurrently (one launch)."""
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    h = ctypes.c_void_p()
    _check(load().csgd_graph_batch_create(arr, len(graphs), ctypes.byref(h)))
    return Graph(h, list(graphs))


class Batch:
    """Many solves in one persistent launch with a device work queue
    (csgd_batch_create): solvers[k] runs n_steps[k] steps from its seed and
    writes x to x_out[k] (CUDA float32, or None)."""

    def __init__(self, solvers, n_steps, x_out=None, wait_limit_ns: int = 0,
                 stall_last_task: bool = False):
        n = len(solvers)
        outs = list(x_out) if x_out is not None else [None] * n
        hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
        st = (ctypes.c_int64 * n)(*[int(k) for k in n_steps])
        xs = (ctypes.c_void_p * n)(*[(_dev_ptr(x, "x_out", sv.part.n_voxels).value if x is not None
                                      else None) for x, sv in zip(outs, solvers)])
        prm = BatchParams(int(wait_limit_ns), int(bool(stall_last_task)), 0)
        h = ctypes.c_void_p()
        _check(load().csgd_batch_create(hs, st, xs, n, ctypes.byref(prm), ctypes.byref(h)))
        self.handle = h
        self._keep = [solvers, outs]

    def launch(self, stream=None):
        _check(load().csgd_batch_launch(self.handle, _stream(stream)))

    def status(self):
        """Waits for the last launch; raises CsgdError (CSGD_ERR_TIMEOUT) if a wait ran out."""
        _check(load().csgd_batch_status(self.handle))

    def info(self) -> dict:
        nt, gr, nu = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        _check(load().csgd_batch_info(self.handle, ctypes.byref(nt), ctypes.byref(nu), ctypes.byref(gr)))
        return dict(tasks=nt.value, units=nu.value, blocks=gr.value)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.csgd_batch_destroy(self.handle)
            self.handle = None


def batch_create(solvers, n_steps, x_out=None, **kw) -> Batch:
    return Batch(solvers, n_steps, x_out, **kw)


def solver_create(part: Partition, params: dict, y, stream=None) -> Solver:
    return Solver(part, params, y, stream)


def solve_step(solver: Solver, j=None, row_blocks=None, stream=None) -> dict:
    return solver.step(j, row_blocks, stream)


def solve(solver: Solver, n_steps: int, x_out=None, report=True, residual=False, stream=None):
    return solver.solve(n_steps, x_out, report, residual, stream)
