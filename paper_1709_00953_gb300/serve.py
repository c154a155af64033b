"""Serving: reconstruction jobs that arrive over time, continuously batched on one GPU.

A job is one scan to reconstruct (geometry, partition, solver settings, data,
number of block steps).  The server keeps every running job's sinogram, volume,
residual and z store resident on the device and admits waiting jobs, in
arrival order, as soon as a slot is free and their device footprint
(``csgd_solver_footprint_bytes`` plus the job's own buffers) fits in the HBM
budget.  Each admitted job runs on its own CUDA stream, so its kernels overlap
with those of the jobs already running; completion is detected with CUDA
events and the job's memory is released for the next ones.  Latency is
measured from arrival to the job's result being on the host.

The host work of a job runs on a small pool of worker threads, not on the
loop that admits and retires jobs: on arrival, its geometry, partition (the
P(I,J) table) and footprint; on admission, the upload of its data, the
solver's allocation and the launch of its solve.  The library's calls release
the interpreter lock, so this work overlaps the loop and the other jobs' host
work.

The kernels are deterministic and jobs share no state, so a job's result is
the same whether it runs alone or in the mix.
"""
from __future__ import annotations

import concurrent.futures as cf
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import csgd


@dataclass
class Job:
    cfg: dict
    y: np.ndarray                 # host sinogram (FP32)
    arrival: float = 0.0          # seconds after the start of the run
    name: str = ""
    # filled by the server
    admitted: float = -1.0
    done: float = -1.0
    x: np.ndarray | None = None
    footprint: int = 0
    latency: float = field(default=-1.0)


class _Prepared:
    """A job's host-side objects, built on arrival: geometry, partition, footprint."""

    def __init__(self, job: Job):
        cfg = job.cfg
        self.geometry = csgd.Geometry(cfg["geom"])
        self.partition = csgd.Partition(self.geometry, **cfg["part"])
        self.footprint = (csgd.footprint_bytes(self.partition, cfg["solver"])
                          + 4 * (self.partition.n_rays + self.partition.n_voxels))


class _Running:
    """An admitted job: data uploaded, solver allocated, whole solve enqueued on
    its stream, followed by x to pinned host memory and an event."""

    def __init__(self, job: Job, prep: _Prepared, stream: torch.cuda.Stream):
        self.job = job
        self.stream = stream
        self.prep = prep
        cfg = job.cfg
        with torch.cuda.stream(stream):
            y_host = torch.from_numpy(np.ascontiguousarray(job.y, np.float32)).pin_memory()
            self.y = torch.empty(y_host.numel(), dtype=torch.float32, device="cuda")
            self.y.copy_(y_host, non_blocking=True)
            self._y_host = y_host
            self.solver = csgd.Solver(prep.partition, cfg["solver"], self.y, stream=stream)
            self.x_host = torch.empty(prep.partition.n_voxels, dtype=torch.float32).pin_memory()
            self.solver.solve(int(cfg["steps"]), self.x_host, report=False, stream=stream)
            self.event = torch.cuda.Event()
            self.event.record(stream)

    def finished(self) -> bool:
        return self.event.query()


def job_footprint(cfg: dict) -> int:
    """Device bytes a job holds while it runs (solver state, data, output)."""
    return _Prepared(Job(cfg, np.zeros(0, np.float32))).footprint


class Server:
    """Continuous batching of reconstruction jobs within an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, max_running: int = 16, workers: int = 4):
        self.budget = int(hbm_budget_bytes)
        self.max_running = int(max_running)
        self.workers = int(workers)
        self.streams = [torch.cuda.Stream() for _ in range(self.max_running)]
        self.max_concurrency = 0
        self.max_used = 0

    def run(self, jobs: list[Job], poll_s: float = 1e-4) -> list[Job]:
        """Serve the jobs (arrival times relative to now); returns them completed."""
        waiting = sorted(jobs, key=lambda j: j.arrival)
        preparing: dict[int, cf.Future] = {}  # id(job) -> _Prepared, from arrival on
        starting: list[tuple[Job, cf.Future]] = []  # admitted, set-up in progress
        running: list[_Running] = []
        free_streams = list(self.streams)
        used = 0
        # Finished jobs' device objects are released in batches, not one by
        # one: freeing device memory waits for the whole device, which would
        # stall the loop behind every running job.  Their bytes count against
        # the budget until they are released.
        retired: list[_Running] = []
        retired_bytes = 0
        device = torch.cuda.current_device()

        def on_worker(fn, *a):
            def call():
                torch.cuda.set_device(device)
                return fn(*a)
            return pool.submit(call)

        with cf.ThreadPoolExecutor(max_workers=self.workers) as pool:
            t0 = time.perf_counter()
            while waiting or starting or running:
                now = time.perf_counter() - t0
                # set-ups that finished become running jobs
                for item in list(starting):
                    if item[1].done():
                        running.append(item[1].result())
                        starting.remove(item)
                # completions: they free streams (and, once released, memory)
                for r in list(running):
                    if r.finished():
                        r.job.done = time.perf_counter() - t0
                        r.job.latency = r.job.done - r.job.arrival
                        r.job.x = r.x_host.numpy().copy()
                        retired_bytes += r.job.footprint
                        free_streams.append(r.stream)
                        running.remove(r)
                        retired.append(r)
                # arrived jobs get their host-side objects built on the workers
                for j in waiting:
                    if j.arrival > now:
                        break
                    if id(j) not in preparing:
                        preparing[id(j)] = on_worker(_Prepared, j)
                # admissions in arrival order while the head job fits
                while waiting and waiting[0].arrival <= now and free_streams:
                    job = waiting[0]
                    fut = preparing[id(job)]
                    if not fut.done():
                        break
                    prep = fut.result()
                    job.footprint = prep.footprint
                    if job.footprint > self.budget:
                        raise ValueError("job %s needs %d bytes, more than the budget"
                                         % (job.name, job.footprint))
                    if used + job.footprint > self.budget:
                        if not retired:
                            break
                        retired.clear()  # releases their device memory
                        used -= retired_bytes
                        retired_bytes = 0
                        continue
                    waiting.pop(0)
                    del preparing[id(job)]
                    job.admitted = time.perf_counter() - t0
                    used += job.footprint
                    starting.append((job, on_worker(_Running, job, prep, free_streams.pop())))
                    self.max_concurrency = max(self.max_concurrency, len(running) + len(starting))
                    self.max_used = max(self.max_used, used)
                if waiting or starting or running:
                    time.sleep(poll_s)
        retired.clear()
        return jobs


def summary(jobs: list[Job], wall_s: float) -> dict:
    lat = np.array([j.latency for j in jobs])
    return {"jobs": len(jobs), "solves_per_s": len(jobs) / wall_s,
            "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean())}


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process with the given rate (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))
