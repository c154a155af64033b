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

The kernels are deterministic and jobs share no state, so a job's result is
the same whether it runs alone or in the mix.
"""
from __future__ import annotations

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


class _Running:
    def __init__(self, job: Job, stream: torch.cuda.Stream):
        self.job = job
        self.stream = stream
        cfg = job.cfg
        with torch.cuda.stream(stream):
            self.geometry = csgd.Geometry(cfg["geom"])
            self.partition = csgd.Partition(self.geometry, **cfg["part"])
            y_host = torch.from_numpy(np.ascontiguousarray(job.y, np.float32)).pin_memory()
            self.y = torch.empty(y_host.numel(), dtype=torch.float32, device="cuda")
            self.y.copy_(y_host, non_blocking=True)
            self._y_host = y_host
            self.solver = csgd.Solver(self.partition, cfg["solver"], self.y, stream=stream)
            self.x_host = torch.empty(self.partition.n_voxels, dtype=torch.float32).pin_memory()
            self.solver.solve(int(cfg["steps"]), self.x_host, report=False, stream=stream)
            self.event = torch.cuda.Event()
            self.event.record(stream)

    def finished(self) -> bool:
        return self.event.query()


def job_footprint(cfg: dict) -> int:
    """Device bytes a job holds while it runs (solver state, data, output)."""
    g = csgd.Geometry(cfg["geom"])
    p = csgd.Partition(g, **cfg["part"])
    return csgd.footprint_bytes(p, cfg["solver"]) + 4 * (p.n_rays + p.n_voxels)


class Server:
    """Continuous batching of reconstruction jobs within an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, max_running: int = 16):
        self.budget = int(hbm_budget_bytes)
        self.max_running = int(max_running)
        self.streams = [torch.cuda.Stream() for _ in range(self.max_running)]
        self.max_concurrency = 0
        self.max_used = 0

    def run(self, jobs: list[Job], poll_s: float = 2e-4) -> list[Job]:
        """Serve the jobs (arrival times relative to now); returns them completed."""
        for j in jobs:
            j.footprint = job_footprint(j.cfg)
            if j.footprint > self.budget:
                raise ValueError("job %s needs %d bytes, more than the budget" % (j.name, j.footprint))
        waiting = sorted(jobs, key=lambda j: j.arrival)
        running: list[_Running] = []
        free_streams = list(self.streams)
        used = 0
        # Finished jobs' device objects are released in batches, not one by
        # one: freeing device memory waits for the whole device, which would
        # stall the loop behind every running job.  Their bytes count against
        # the budget until they are released.
        retired: list[_Running] = []
        retired_bytes = 0
        t0 = time.perf_counter()
        while waiting or running:
            now = time.perf_counter() - t0
            # completions first: they free streams (and, once released, memory)
            for r in list(running):
                if r.finished():
                    r.job.done = time.perf_counter() - t0
                    r.job.latency = r.job.done - r.job.arrival
                    r.job.x = r.x_host.numpy().copy()
                    retired_bytes += r.job.footprint
                    free_streams.append(r.stream)
                    running.remove(r)
                    retired.append(r)
            # admissions in arrival order while the head job fits
            while waiting and waiting[0].arrival <= now and free_streams:
                if used + waiting[0].footprint > self.budget:
                    if not retired:
                        break
                    retired.clear()  # releases their device memory
                    used -= retired_bytes
                    retired_bytes = 0
                    continue
                job = waiting.pop(0)
                job.admitted = time.perf_counter() - t0
                used += job.footprint
                running.append(_Running(job, free_streams.pop()))
                self.max_concurrency = max(self.max_concurrency, len(running))
                self.max_used = max(self.max_used, used)
            if waiting or running:
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
