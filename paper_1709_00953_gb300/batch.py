"""Many independent problems solved together.

Each problem keeps its own geometry, partition and solver state on the device.
Three ways to run a set of problems:

* ``Batch.launch`` (the batched form): every block step of every problem in
  ONE persistent kernel launch with a device work queue (csgd_batch_create):
  the kernels of all solves become tasks of thread blocks, interleaved across
  problems; executor blocks take work from a ticket counter and wait (bounded)
  for their problem's earlier kernels.  The launch is captured in a CUDA graph
  with the problems' resets.
* ``Batch.launch_graphs``: a graph whose child graphs are the problems' solves
  (each captured once, launch shapes optionally autotuned for its sizes), with
  no dependencies between them, so the GPU overlaps them.
* ``Batch.launch_sequential_graphs`` / ``Batch.solve_one_by_one``: the same
  solve graphs launched one after the other, or the plain host-launched solves
  with a synchronisation after each problem: the baselines.

The kernels are deterministic and the problems share no state, so the graph
forms equal the one-by-one solves bit for bit; the executor runs the same
kernel bodies with one lane per ray and 256-thread blocks and agrees with them
to rounding.
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
        self.shapes = (0, 0)
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
    """A set of problems, their solve graphs and the persistent batch launch."""

    def __init__(self, problems, autotune: bool = False, executor: bool = True,
                 graphs: bool = True, wait_limit_ns: int = 0):
        self.problems = list(problems)
        if autotune:
            for p in self.problems:
                p.autotune()
        # the graphs are captured first: capturing plans each solver afresh
        self.graph = csgd.graph_batch([p.graph() for p in self.problems]) if graphs else None
        self.executor = (csgd.Batch([p.solver for p in self.problems], [p.steps for p in self.problems],
                                    [p.x for p in self.problems], wait_limit_ns=wait_limit_ns)
                         if executor else None)

    def launch(self, stream=None):
        """All problems in one persistent launch (the executor)."""
        self.executor.launch(stream)

    def status(self):
        """Waits for the last executor launch; raises if one of its waits ran out."""
        self.executor.status()

    def launch_graphs(self, stream=None):
        """All problems' solve graphs as children of one graph, overlapped."""
        self.graph.launch(stream)

    def launch_sequential_graphs(self, stream=None):
        """The same solve graphs, one after the other on one stream."""
        for p in self.problems:
            p.graph().launch(stream)

    def solve_one_by_one(self, stream=None):
        for p in self.problems:
            p.solve_plain(stream)
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
