"""Benchmark of the CSGD / GCSGD block solver on GB300.

One bench step = one complete solve of the workload (solver state reset to
x = 0, z = 0, r = y, then every block step of the workload, its residual
refreshes and epoch averages).  The default workload is the paper-scale 3D
cone beam (256^3 voxels, 360 views x 384^2 pixels, 360 single-view row blocks
x 4 x 4 x 4 tiles, groups of 30 views drawn by density: one epoch = 768 group
steps, Alg. 4).

metric: ray-voxel updates/s, where one update applies one non-zero A_ij of the
block to one vector: every step does one backprojection and two forward
products, so updates = 3 * nnz(A_{I_g}^J), counted by the kernels.

roofline: the dominant kernel's algorithmic bytes (what the method itself must
move for it, per step: backprojection r in on the step's rays R and g out on
the tile's voxels |J|, 4 (R + |J|) bytes; dual forward x_J and g_J in, p and q
out, 4 (2 |J| + 2 R) bytes) per second, against the measured HBM copy rate.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                        [--workload cone3d_256|fan2d_512|parallel2d_64|batch_fan64|serve]
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synth import configs as C  # noqa: E402
from synth import data as D  # noqa: E402

# Ray-voxel updates per non-zero of A_{I_g}^J for each timed kernel.
UPDATES_PER_NNZ = {"backproject": 1, "forward_dual": 2}
# enough solves for a timed region of about 1 s (several clock samples)
DEFAULT_STEPS = {"fan2d_512": 250, "parallel2d_64": 250, "cone3d_256": 16, "batch_fan64": 20}
DEFAULT_WORKLOAD = "cone3d_256"


def algorithmic_bytes(kernel: str, rays: int, tile_voxels: int, batch_voxels: int | None = None,
                      volume_voxels: int = 0, epoch_rays: int = 0) -> int:
    """Bytes a kernel unit must move by the method's own definition (FP32), for
    steps covering `rays` rays of their row blocks (in tile J's shadow) and
    `tile_voxels` voxels of their tiles: the backprojection reads r and writes
    g; the dual forward reads x_J and g_J and writes p and q; the epilogue
    reads p, q, z and r and writes z and r per ray, reads g_J per step and, once
    per batch of steps on one tile (`batch_voxels` = the batches' tile voxels,
    default one batch per step), reads x_J and updates x^_J; the epoch close
    reads x^ and writes x and x^ over `volume_voxels` (and, under epoch sync,
    reads the pending change and r and writes r over `epoch_rays`)."""
    if kernel == "backproject":
        return 4 * (rays + tile_voxels)
    if kernel == "forward_dual":
        return 4 * (2 * rays + 2 * tile_voxels)
    if kernel == "epilogue":
        bv = tile_voxels if batch_voxels is None else batch_voxels
        return 4 * (6 * rays + tile_voxels + 3 * bv)
    if kernel == "epoch_close":
        return 4 * (3 * volume_voxels + 3 * epoch_rays)
    return 0


# Per launch of a kernel unit, from one ncu capture of the workload with the
# kernel sources of the given hash (ops.cu, device.cuh, common.h without
# comments): dram__bytes_read.sum + dram__bytes_write.sum ("traffic") and
# sm__instruction_throughput (the issue slots used, % of peak).  A kernel
# edit changes the hash and voids the entry ("traffic" is then null).
# "backproject" is the ray table plus the gather, or the ray table, the scatter
# and its conversion pass: the unit the bench times.
NCU_COUNTERS: dict = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,
    #   smsp__issue_active.avg.pct_of_peak_sustained_active,
    #   sm__throughput.avg.pct_of_peak_sustained_elapsed,gpu__time_duration.sum
    #   --clock-control none -k regex:"k_slot_rmax|k_backproject_scatter|k_scatter_convert|
    #   k_forward_dual|k_epilogue" -s 10 -c 10 python bench.py --no-cpu --no-e2e --no-extras
    #   --steps 1 --warmup 3 --launch=-1,1  (GB300; mean of two batches of 12 slots);
    # the L2 figures from ncu --set full -k regex:"k_forward_dual|k_backproject_scatter"
    # -s 6 -c 2 on the same command
    ("cone3d_256_360x384x384_360x64_g30", "1922eec259ea1d80"): {
        "backproject": {"traffic": 55566000, "issue_active_pct": 60.0,
                        "lts_throughput_pct": 82.0, "l2_atomic_input_active_pct": 58.8,
                        "parts": "max |r| pass 14.6 MB + scatter 27.3 MB + conversion 13.6 MB"},
        "forward_dual": {"traffic": 28032000, "issue_active_pct": 71.3},
    },
}
KERNEL_SOURCES = ("paper_1709_00953_gb300/csrc/ops.cu", "paper_1709_00953_gb300/csrc/device.cuh",
                  "paper_1709_00953_gb300/csrc/common.h")


def kernel_hash() -> str:
    """Hash of the kernel sources without comments and blank lines: a change
    of the code voids the stored traffic figures, a change of a comment not."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        lines = [ln.rstrip() for ln in src.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 16 solves of cone3d_256, more for the smaller workloads)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(C.ALL) + ["batch_fan64", "serve"])
    ap.add_argument("--rate", type=float, default=200.0, help="serve: arrivals per second")
    ap.add_argument("--jobs", type=int, default=40, help="serve: number of requests")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and served forms reported beside the headline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's launch-shape models instead of csgd_solver_autotune")
    ap.add_argument("--launch", default=None,
                    help="fixed launch shapes, --launch=bp_groups,fwd_lanes (bp_groups -1: scatter, "
                         "-2: bricks) instead of csgd_solver_autotune")
    a = ap.parse_args()
    if a.steps is None:
        a.steps = DEFAULT_STEPS.get(a.workload, 20)
    return a


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
class OracleSteps:
    """The FP64 oracle's block steps of a workload's schedule, one at a time.

    A step is one Alg. 1 step of the schedule.  For grouped workloads (Alg. 4,
    a group of s row blocks per step) one oracle step of a full group takes
    tens of seconds on the host, so there a step is the Alg. 1 step on one row
    block of the scheduled group (the group's blocks in turn): a bounded
    sample with the same per-update work."""

    def __init__(self, cfg, y):
        from oracle.blocks import Partition as OPart
        from oracle.geometry import Geometry as OGeom
        from oracle.solver import OracleSolver
        og = OGeom(**cfg["geom"])
        self.op = OPart(og, cfg["part"]["tiles"], cfg["part"]["view_blocks"],
                        cfg["part"]["det_blocks"])
        self.o = OracleSolver(self.op, cfg["solver"], np.asarray(y, np.float64))
        self.grouped = int(cfg["solver"].get("group_size", 1)) > 1
        self.pending = []

    def next(self):
        if not self.pending:
            if not self.o.queue:
                self.o._new_epoch()
            j, grp, _ = self.o.queue.pop(0)
            self.pending = [(j, [i]) for i in grp] if self.grouped else [(j, list(grp))]
        return self.pending.pop(0)

    def step(self):
        """One step: (seconds, non-zeros of its block)."""
        from oracle.blocks import block_nnz
        j, grp = self.next()
        t0 = time.perf_counter()
        self.o.step(j, grp)
        dt = time.perf_counter() - t0
        return dt, block_nnz(self.op, grp, j)

    def what(self) -> str:
        return ("Alg. 1 steps on single row blocks of the scheduled groups" if self.grouped
                else "scheduled block steps (Alg. 1)")


def oracle_sample(cfg, y, seconds: float, max_steps: int | None = None):
    """Time the oracle's steps (see OracleSteps) for about `seconds`."""
    from oracle import siddon
    st = OracleSteps(cfg, y)
    spent, steps, nnz = 0.0, 0, 0
    while max_steps is None or steps < max_steps:
        dt, nz = st.step()
        spent += dt
        nnz += nz
        steps += 1
        if spent >= seconds:
            break
    return dict(seconds=spent, steps=steps, nnz=nnz, cores=siddon.num_threads(), what=st.what())


def run_reference(args, cfg, world, rank):
    """--impl reference: the FP64 oracle, on the host cores, on this workload."""
    if rank != 0:
        return 0
    big = cfg["geom"]["kind"] == "cone3d"
    y, _ = D.make_data(cfg, device="cuda" if big and _cuda_ok() else None)
    st = OracleSteps(cfg, y)
    for _ in range(args.warmup):
        st.step()
    t = 0.0
    nnz = 0
    for _ in range(args.steps):
        dt, nz = st.step()
        t += dt
        nnz += nz
    from oracle import siddon
    og = st.op.geom
    value = 3.0 * nnz / t
    line = {
        "impl": "reference", "metric": "ray-voxel updates/s", "value": value,
        "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "block_steps_per_solve": int(cfg["steps"]),
                   "n_rays": int(og.n_rays), "n_voxels": int(og.grid.size),
                   "parallelism": "host cores (FP64 oracle)",
                   "step": "one %s, a bounded sample of the workload's solve"
                           % st.what().replace("steps", "step", 1)},
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": siddon.num_threads(),
                         "kind": "oracle",
                         "sample": "%d %s of %s after %d warm-up steps"
                                   % (args.steps, st.what(), cfg["name"], args.warmup)},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _cuda_ok() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# ---------------------------------------------------------------------------
# multi-rank timing (replicas: every rank solves its own copy of the workload)
# ---------------------------------------------------------------------------
def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The largest of the ranks' times (every rank gets it): the job's time."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms / 1e3)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, cfg, world, rank, local):
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__ as GE
    GE.build()
    from paper_1709_00953_gb300 import csgd

    big = cfg["geom"]["kind"] == "cone3d"
    y, _ = D.make_data(cfg, device=str(dev) if big else None)
    g = csgd.Geometry(cfg["geom"])
    p = csgd.Partition(g, **cfg["part"])
    yt = torch.tensor(y, device=dev)
    stream = torch.cuda.current_stream()
    solver = csgd.Solver(p, cfg["solver"], yt)
    if args.launch:
        solver.set_launch(*(int(v) for v in args.launch.split(",")))
    steps = cfg["steps"]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def one_solve_direct():
        solver.reset(yt)
        solver.solve(steps, None, report=False)

    for _ in range(args.warmup):
        one_solve_direct()
    rep = None
    solver.reset(yt)
    rep = solver.solve(steps, None, report=True)
    nnz_per_solve = rep["nnz"]
    torch.cuda.synchronize()
    # launch shapes for this workload (csgd_solver_autotune, which resets the
    # solver), then the solve as one CUDA graph (reset, every block step, epoch
    # averages): the library's path for repeated solves
    if args.launch:
        shapes = tuple(int(v) for v in args.launch.split(","))
        solver.set_launch(*shapes)
    else:
        shapes = None if args.no_autotune else solver.autotune(min(steps, 16))
    graph = solver.graph(steps)

    def one_solve():
        graph.launch()

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident, L2 flushed before every step ----
    def timed(instrumented: bool, fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(torch.cuda.current_device())
        solver.profile(instrumented)
        solver.profile_read(reset=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ck = clocks.stop()
        prof = solver.profile_read(reset=True)
        solver.profile(False)
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world, dev)
        if world > 1:
            torch.distributed.barrier()
        return ms, wall, ck, prof

    # the headline: graph launches, no per-kernel events in the stream
    ms, t_wall, ck, _ = timed(False, one_solve)
    # the same K solves launched kernel by kernel with CUDA events around every
    # launch, on the solver's stream: per-kernel durations for the roofline and
    # the shares
    ms_instr, _, _, prof = timed(True, one_solve_direct)
    value = job_rate(3.0 * nnz_per_solve * args.steps, world, ms)

    # ---- end to end through the public API: pinned host y in, host x out ----
    e2e = None
    if not args.no_e2e:
        y_host = torch.tensor(y).pin_memory()
        x_host = torch.empty(p.n_voxels, dtype=torch.float32).pin_memory()
        # y from pinned host memory into the solver (csgd_solver_reset), then the
        # solve graph, which ends with x copied to pinned host memory
        graph_e2e = solver.graph(steps, x_host)
        for _ in range(2):
            solver.reset(y_host)
            graph_e2e.launch()
        torch.cuda.synchronize()
        e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            e_ev[k][0].record(stream)
            solver.reset(y_host)
            graph_e2e.launch()
            e_ev[k][1].record(stream)
            torch.cuda.synchronize()
        e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e_ev), world, dev)
        e2e = {"value": job_rate(3.0 * nnz_per_solve * args.steps, world, e_ms), "unit": "updates/s",
               "h2d_bytes_per_step": int(4 * p.n_rays), "d2h_bytes_per_step": int(4 * p.n_voxels),
               "ms_per_step": e_ms / args.steps}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel ----
    # algorithmic bytes (see algorithmic_bytes) of the kernel over the timed
    # solves, per launch, against the measured HBM copy rate
    kern = {k: v for k, v in prof.items() if v["launches"] > 0}
    total_ms = sum(v["ms"] for v in kern.values())
    dom = max(("backproject", "forward_dual"), key=lambda k: kern.get(k, {"ms": 0})["ms"])
    dom_s = kern[dom]["ms"] / 1e3
    n_launch = int(kern[dom]["launches"])
    nnz_total = nnz_per_solve * args.steps
    alg_launch = algorithmic_bytes(dom, rep["rays"], rep["tile_voxels"]) * args.steps / n_launch
    achieved = alg_launch * n_launch / dom_s / 1e9
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    basis = "measured HBM copy rate (MEASURED_PEAKS.json hbm_gbs)"
    if not hbm:
        hbm, basis = 6800.0, "fallback HBM figure (no measured peaks file)"
    counters = NCU_COUNTERS.get((cfg["name"], kernel_hash()), {}).get(dom, {})
    traffic = counters.get("traffic")
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "peak_basis": basis,
            "algorithmic_bytes_per_launch": alg_launch, "kernel_launches": n_launch,
            "ms_per_launch": kern[dom]["ms"] / n_launch,
            "algorithmic_bytes_basis": "per step: backprojection 4 (R + |J|), dual forward "
                                       "4 (2 R + 2 |J|) (R rays of the step's row blocks in "
                                       "tile J's shadow, |J| voxels of the tile)",
            "updates_per_s": UPDATES_PER_NNZ[dom] * nnz_total / dom_s,
            "csr_equivalent_gbs": 8.0 * nnz_total / dom_s / 1e9,
            "csr_equivalent_note": "avoided work: the bytes a stored-matrix SpMV (FP32 value + int32 "
                                   "index per non-zero) would stream for the same non-zeros"}
    if traffic is not None:
        roof["dram_gbs"] = traffic * n_launch / dom_s / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / hbm
        roof["traffic_over_algorithmic"] = traffic / alg_launch
    for key in ("issue_active_pct", "lts_throughput_pct", "l2_atomic_input_active_pct"):
        if counters.get(key) is not None:
            roof[key] = counters[key]
    # the HBM-bound kernels (the z and r update with the x^ accumulation, and the
    # epoch close) against the same roof, on their algorithmic bytes
    hbm_k = {}
    n_epi = int(prof["epilogue"]["launches"])
    if n_epi:
        batch_vox = rep["tile_voxels"] * (n_epi / args.steps) / steps
        b = algorithmic_bytes("epilogue", rep["rays"], rep["tile_voxels"], batch_vox) * args.steps / n_epi
        t = prof["epilogue"]["ms"] / n_epi / 1e3
        hbm_k["epilogue"] = {"algorithmic_bytes_per_launch": b, "ms_per_launch": t * 1e3,
                             "achieved_gbs": b / t / 1e9, "frac": b / t / 1e9 / hbm}
    n_close = int(prof["epoch_close"]["launches"])
    if n_close:
        sync_epoch = cfg["solver"].get("sync", 0) == 1
        b = algorithmic_bytes("epoch_close", 0, 0, volume_voxels=p.n_voxels,
                              epoch_rays=p.n_rays if sync_epoch else 0)
        t = prof["epoch_close"]["ms"] / n_close / 1e3
        hbm_k["epoch_close"] = {"algorithmic_bytes_per_launch": b, "ms_per_launch": t * 1e3,
                                "achieved_gbs": b / t / 1e9, "frac": b / t / 1e9 / hbm}
    roof["hbm_kernels"] = hbm_k
    # the whole step against the same roof: compulsory bytes 4 (2 R + 3 |J|) per step (r of the
    # shadow rays in, z out, x_J in, x^_J in and out)
    step_bytes = 4 * (2 * rep["rays"] + 3 * rep["tile_voxels"]) * args.steps
    roof["step_bytes_gbs"] = step_bytes / (ms / 1e3) / 1e9
    # per batch: the backprojection (ray table + gather; max |r| pass + scatter +
    # conversion; or one brick kernel), dual forward, epilogue; per epoch close:
    # averaging (+ pending-residual apply under epoch sync)
    close_kernels = 2 if cfg["solver"].get("sync", 0) == 1 else 1
    bp_form = shapes[0] if shapes else 0
    bp_kernels = 3 if bp_form == csgd.SCATTER else (1 if bp_form in csgd.BRICKS else 2)
    launches = int(bp_kernels * prof["backproject"]["launches"] + prof["forward_dual"]["launches"]
                   + prof["epilogue"]["launches"] + close_kernels * prof["epoch_close"]["launches"])
    kernels = {k: {"launches": int(v["launches"]), "ms": v["ms"],
                   "share": (v["ms"] / total_ms if total_ms else 0.0)} for k, v in kern.items()}

    cpu = None
    if not args.no_cpu:
        res = oracle_sample(cfg, y, seconds=args.cpu_seconds)
        cpu = {"value": 3.0 * res["nnz"] / res["seconds"], "unit": "updates/s",
               "cores": res["cores"], "kind": "oracle",
               "steps_per_s": res["steps"] / res["seconds"],
               "sample": "first %d %s of %s (%.1f s of FP64 oracle work)"
                         % (res["steps"], res["what"], cfg["name"], res["seconds"])}
        # the same oracle on one host core, a shorter sample (skipped where one
        # block step alone would take too long on one core)
        from oracle import siddon
        n_all = siddon.num_threads()
        if res["seconds"] / max(1, res["steps"]) * min(n_all, 8) <= args.cpu_seconds:
            siddon.set_threads(1)
            try:
                one = oracle_sample(cfg, y, seconds=args.cpu_seconds / 3)
            finally:
                siddon.set_threads(n_all)
            cpu["value_1core"] = 3.0 * one["nnz"] / one["seconds"]
            cpu["sample_1core"] = "first %d %s (%.1f s)" % (one["steps"], one["what"], one["seconds"])
        else:
            cpu["value_1core"] = None
            cpu["sample_1core"] = "skipped: one step exceeds the sample budget on one core"

    line = {
        "metric": "ray-voxel updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": cfg["name"], "block_steps_per_solve": steps,
                   "nnz_per_solve": int(nnz_per_solve), "n_rays": int(p.n_rays),
                   "n_voxels": int(p.n_voxels), "l2": "flushed (256 MB write) before each step",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "solves_per_s": 1e3 * args.steps * world / ms,
                   "epochs_per_solve": int(rep["epochs"]),
                   "ms_per_epoch": ms / args.steps / max(1, int(rep["epochs"]))},
        "roofline": roof, "kernels": kernels, "gpu_launches": launches,
        "launch": "one CUDA graph per solve (reset, all block steps, epoch averages)",
        "launch_shapes": ({"autotuned": not args.launch,
                           "backprojection": "scatter" if shapes[0] == csgd.SCATTER else (
                               "brick" if shapes[0] in csgd.BRICKS else "gather"),
                           "view_groups": shapes[0], "lanes_per_ray": shapes[1]}
                          if shapes else {"autotuned": False}),
        "kernel_timing": "per-launch CUDA events in a second pass of the same %d solves launched "
                         "kernel by kernel (%.3f ms per solve that way)" % (args.steps, ms_instr / args.steps),
        "wall_s_timed": t_wall,
    }
    if ck:
        line["clocks"] = ck
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = cpu
    if world == 1 and not args.no_extras:
        # the batched (64 uneven fans) and served (Poisson mix) forms, in the same
        # run: their own short timings, reported beside the headline
        line["also"] = {}
        for name, fn in (("batch_fan64", run_batch), ("serve", run_serve)):
            sub = argparse.Namespace(**vars(args))
            sub.steps, sub.warmup = (6, 1) if name == "batch_fan64" else (args.steps, 2)
            try:
                r = fn(sub, world, rank, local, emit=False)
                keep = ("metric", "value", "unit", "ms_per_step", "config", "forms", "speedup_vs_one_by_one",
                        "speedup_vs_sequential_graphs", "equal_rmse", "latency", "capacity",
                        "one_at_a_time", "served_equals_one_at_a_time", "max_concurrency", "executor",
                        "clocks")
                line["also"][name] = {k: r[k] for k in keep if k in r}
            except Exception as ex:  # reported, never fatal to the headline
                line["also"][name] = {"error": repr(ex)[:300]}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# batched workload: 64 uneven fan problems, one graph launch vs one by one
# ---------------------------------------------------------------------------
def run_batch(args, world, rank, local, emit=True):
    # a single-GPU workload: under torchrun rank 0 runs it and the others exit
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local if world > 1 else 0)
    import __graft_entry__ as GE
    GE.build()
    from paper_1709_00953_gb300 import batch
    cfgs = C.batch_fan2d()
    probs = [batch.Problem(c, D.make_data(c, device="cuda")[0]) for c in cfgs]
    t_tune = time.perf_counter()
    b = batch.Batch(probs, autotune=True)
    t_tune = time.perf_counter() - t_tune
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def executor():
        b.launch(stream)

    forms = {"persistent": executor, "graph_of_graphs": lambda: b.launch_graphs(stream),
             "sequential_graphs": lambda: b.launch_sequential_graphs(stream),
             "one_by_one": lambda: b.solve_one_by_one(stream)}
    for _ in range(args.warmup):
        for fn in forms.values():
            fn()
        b.status()
    torch.cuda.synchronize()
    # updates per round (kernel-counted non-zeros of every problem's solve)
    nnz = 0
    for p in probs:
        p.solver.reset(p.y)
        rep = p.solver.solve(p.steps, p.x, report=True)
        nnz += rep["nnz"]
    torch.cuda.synchronize()

    def timed(fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            fn()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in ev)

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms = {"persistent": timed(executor)}
    ck = clocks.stop()
    b.status()
    x_exec = [p.x.clone() for p in probs]
    for name in ("graph_of_graphs", "sequential_graphs", "one_by_one"):
        ms[name] = timed(forms[name])
    x_plain = [p.x.clone() for p in probs]
    b.launch_graphs(stream)
    torch.cuda.synchronize()
    graphs_equal = all(torch.equal(p.x, x) for p, x in zip(probs, x_plain))
    # the executor's solutions against the one-by-one ones (the same RMSE to rounding)
    rel = max(float(torch.sqrt(torch.mean((xe.double() - xp.double()) ** 2)))
              / max(float(xp.abs().max()), 1e-30) for xe, xp in zip(x_exec, x_plain))
    n = len(probs)
    rate = {k: 1e3 * n * args.steps / v for k, v in ms.items()}
    info = b.executor.info()
    line = {
        "metric": "solves/s at fixed step count (64 uneven fan problems, one persistent launch)",
        "value": rate["persistent"], "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms["persistent"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batch_fan64", "problems": n,
                   "sizes": "n ~ U[128,1024], views ~ U[60,900], 3 epochs each",
                   "l2": "flushed (256 MB write) before each step"},
        "forms": {k: {"solves_per_s": rate[k], "ms_per_step": ms[k] / args.steps} for k in ms},
        "speedup_vs_one_by_one": ms["one_by_one"] / ms["persistent"],
        "speedup_vs_sequential_graphs": ms["sequential_graphs"] / ms["persistent"],
        "updates_per_s": 3.0 * nnz * args.steps / (ms["persistent"] / 1e3),
        "executor": dict(info, note="tasks = the kernels of all solves; units = their thread "
                                    "blocks; blocks = resident executor blocks"),
        "equal_rmse": {"graph_forms_bit_identical_to_one_by_one": graphs_equal,
                       "persistent_max_relative_rmse_vs_one_by_one": rel},
        "launch_shapes": {"autotuned": True, "seconds": t_tune,
                          "view_groups": sorted(collections.Counter(p.shapes[0] for p in probs).items()),
                          "lanes_per_ray": sorted(collections.Counter(p.shapes[1] for p in probs).items()),
                          "persistent": "one lane per ray, 256-thread blocks, 4 view groups"},
    }
    if ck:
        line["clocks"] = ck
    if not emit:
        return line
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# serving workload: Poisson arrivals of mixed fan / cone jobs, continuous batching
# ---------------------------------------------------------------------------
def run_serve(args, world, rank, local, emit=True):
    # a single-GPU workload: under torchrun rank 0 runs it and the others exit
    if rank != 0:
        return 0
    import torch
    torch.cuda.set_device(local if world > 1 else 0)
    import __graft_entry__ as GE
    GE.build()
    from paper_1709_00953_gb300 import serve
    cfgs = C.serving_jobs(n_jobs=args.jobs)
    ys = [D.make_data(c, device="cuda")[0] for c in cfgs]
    budget = 40 << 30
    # warm-up: a few jobs served back to back
    warm = [serve.Job(c, y, 0.0, c["name"]) for c, y in list(zip(cfgs, ys))[:max(1, args.warmup)]]
    serve.Server(budget).run(warm)
    # capacity: every job queued at t = 0 (the server's throughput limit)
    sat = [serve.Job(c, y, 0.0, c["name"]) for c, y in zip(cfgs, ys)]
    t0 = time.perf_counter()
    serve.Server(budget, max_running=16).run(sat)
    cap = serve.summary(sat, time.perf_counter() - t0)
    # the plain form: the same jobs, all queued, solved one at a time
    one = [serve.Job(c, y, 0.0, c["name"]) for c, y in zip(cfgs, ys)]
    t0 = time.perf_counter()
    serve.Server(budget, max_running=1, workers=1).run(one)
    one_s = serve.summary(one, time.perf_counter() - t0)
    same = all(np.array_equal(a.x, b.x) for a, b in zip(sat, one))
    # latency at the configured Poisson arrival rate
    arrivals = serve.poisson_arrivals(len(cfgs), args.rate, seed=1709 + 4)
    jobs = [serve.Job(c, y, float(a), c["name"]) for c, y, a in zip(cfgs, ys, arrivals)]
    srv = serve.Server(budget, max_running=16)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t0 = time.perf_counter()
    srv.run(jobs)
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    s = serve.summary(jobs, wall)
    line = {
        "metric": "solves/s with p50/p99 latency (Poisson arrivals, continuous batching)",
        "value": s["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": len(jobs),
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / len(jobs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve", "jobs": len(jobs), "rate_per_s": args.rate,
                   "mix": "fan 256^2-2048^2 (60-720 views, 2 epochs), cone 128^3-512^3 (60-180 "
                          "views, 1 epoch), sizes log-uniform, 1 in 8 a 100^3 / 4.2M-ray cone",
                   "hbm_budget_gb": budget / 2 ** 30},
        "latency": {"p50_s": s["p50_latency_s"], "p99_s": s["p99_latency_s"],
                    "mean_s": s["mean_latency_s"]},
        "max_concurrency": srv.max_concurrency, "wall_s": wall,
        "arrival_window_s": float(arrivals[-1]),
        "capacity": {"solves_per_s": cap["solves_per_s"], "p50_latency_s": cap["p50_latency_s"],
                     "p99_latency_s": cap["p99_latency_s"],
                     "note": "all jobs queued at t = 0: the throughput limit of the server"},
        "one_at_a_time": {"solves_per_s": one_s["solves_per_s"], "p50_latency_s": one_s["p50_latency_s"],
                          "p99_latency_s": one_s["p99_latency_s"],
                          "note": "all jobs queued at t = 0, one running at a time"},
        "served_equals_one_at_a_time": same,
        "quality": "each job runs its fixed step count (the stopping rule: the served result "
                   "is within RMSE 1e-3 of the FP64 oracle's solution of the same job, checked by "
                   "the GPU tests; served results equal solo solves bit for bit)",
    }
    if ck:
        line["clocks"] = ck
    if not emit:
        return line
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.workload == "batch_fan64":
        return run_batch(args, world, rank, local)
    if args.workload == "serve":
        return run_serve(args, world, rank, local)
    cfg = C.ALL[args.workload]()
    if args.impl == "reference":
        return run_reference(args, cfg, world, rank)
    return run_gpu(args, cfg, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
