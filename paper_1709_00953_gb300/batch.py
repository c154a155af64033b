"""Many independent problems solved together: one CUDA-graph launch for all.

Each problem keeps its own geometry, partition and solver state on the device.
Every problem's whole solve (reset, all block steps, epoch averages, x out) is
captured once into a CUDA graph, optionally after its kernel launch shapes are
autotuned for its sizes; the batch is a graph whose child graphs are
those solves, with no dependencies between them, so one launch runs all block
steps of all problems and the GPU overlaps the small ones.  Results are the
same as solving each problem alone: the kernels are deterministic and the
problems share no state.
"""
from __future__ import annotations

import torch

from . import csgd


class Problem:
    """One problem on the device: geometry, partition, solver and its output x."""

    def __init__(self, cfg: dict, y, device=None):
        self.cfg = cfg
        self.geometry = csgd.Geometry(cfg["geom"])
        self.partition = csgd.Partition(self.geometry, **cfg["part"])
        self.y = torch.as_tensor(y, dtype=torch.float32, device=device or "cuda").contiguous()
        self.solver = csgd.Solver(self.partition, cfg["solver"], self.y)
        self.x = torch.zeros(self.partition.n_voxels, dtype=torch.float32, device=self.y.device)
        self.steps = int(cfg["steps"])
        self._graph = None

    def autotune(self, trial_steps: int | None = None) -> tuple:
        """Picks this problem's kernel launch shapes by timing them (before its graph
        is captured); returns (view groups, lanes per ray)."""
        if self._graph is not None:
            raise RuntimeError("autotune before the graph is captured")
        self.shapes = self.solver.autotune(trial_steps or min(self.steps, 16))
        return self.shapes

    def graph(self) -> csgd.Graph:
        if self._graph is None:
            self._graph = self.solver.graph(self.steps, self.x)
        return self._graph

    def solve_plain(self, stream=None) -> dict:
        """The plain path: reset and csgd_solve on the stream (host-driven launches)."""
        self.solver.reset(self.y, stream=stream)
        return self.solver.solve(self.steps, self.x, report=False, stream=stream)


class Batch:
    """A set of problems and the single graph that solves all of them."""

    def __init__(self, problems, autotune: bool = False):
        self.problems = list(problems)
        if autotune:
            for p in self.problems:
                p.autotune()
        self.graph = csgd.graph_batch([p.graph() for p in self.problems])

    def launch(self, stream=None):
        self.graph.launch(stream)

    def solve_one_by_one(self, stream=None):
        for p in self.problems:
            p.solve_plain(stream)
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
