"""Alg. 1 (basic iteration) inside Alg. 2 / Alg. 3 / Alg. 4, literally, in FP64 (oracle).

Test infrastructure only (see the package docstring).

State (Alg. 2 initialisation): x = 0, every z_I^j = 0, r = y.  One step on a
column block J and a group of row blocks I_g (Alg. 1; Alg. 3 with one block per
group; Alg. 4 in general):

    g_J   = (A_{I_g}^J)^T r_{I_g}                      (Eq. 'direction')
    mu    = beta * g_J^T g_J / ||A_{I_g}^J g_J||^2     (Eq. 'step'; 0 if the norm is 0)
    beta  = b * P_S(I_g, J) / P_T(J)                   (Alg. 3 initialisation)
    x^_J += x_J + mu g_J ;  count_J += 1
    z_I^j = A_I^J (x_J + mu g_J) for every I in I_g     (computed as its own
                                                         forward projection)

x_J itself stays fixed during an epoch; after the row draws of one column block
the residual is refreshed on the rows It that were drawn, r_It = y_It -
sum_j z_It^j (Alg. 2-4; the It restriction is the remark after Alg. 3).  At the
end of the epoch every updated block becomes the mean of its candidates,
x_J = x^_J / count_J, and x^ and the counts are reset (end of the epoch loop of Alg. 2-4).

Readings where the paper is silent:

* "sync": the refresh sits inside the column loop in Alg. 2-4 ("column", the
  default).  The parameter-server description of Sec. II-F also allows all
  column batches of an epoch to read the epoch-start residual with a single
  refresh at the end of the epoch ("epoch").
* A run of n steps that stops inside an epoch closes it (refresh of the rows
  drawn so far, then averaging); the next run starts a fresh epoch.
* A block drawn with zero overlap (possible under uniform sampling) gives
  g = 0, mu = 0 and a candidate equal to x_J, which is counted in the mean.
  More generally mu = 0 whenever A g = 0 (Eq. 'step' is undefined there and
  the step direction has no effect on the block's rows).

Parity: the single-step decrease identity, steepest descent against a dense
least-squares solve (m = n = 1), the m = 1 column-action property (r = y - A x
exactly after every epoch, across tiles), the epoch mean of candidates, and
whole runs with m = 8 row blocks and n = 2 tiles reaching the exact solution of
a consistent full-rank problem (importance and uniform sampling) are pinned in
``tests/test_oracle_solver.py``.  The paper prints no trajectory to compare a
run with step by step.
"""
from __future__ import annotations

import numpy as np

from . import schedule as S
from .blocks import Partition, backproject_block, project_block
from .ptable import probability_table

COLUMN, EPOCH = 0, 1

def step_length(beta: float, gg: float, qq: float) -> float:
    """mu = beta g^T g / ||A g||^2 (Eq. 'step'), and 0 when A g = 0."""
    if qq > 0.0:
        return beta * gg / qq
    return 0.0


def default_params(**kw) -> dict:
    p = dict(sampling=S.IMPORTANCE, alpha=1.0, gamma=1.0, b=1.0, group_size=1,
             sync=COLUMN, seed=0, theta_step=1.0 / 40.0)
    p.update(kw)
    return p


class OracleSolver:
    def __init__(self, part: Partition, params: dict, y: np.ndarray, P: np.ndarray | None = None):
        self.part = part
        self.p = default_params(**params)
        self.P = probability_table(part) if P is None else np.asarray(P, np.float64)
        g = part.geom
        self.y = np.asarray(y, np.float64).reshape(g.n_rays).copy()
        self.x = np.zeros(g.grid.size)
        self.xhat = np.zeros(g.grid.size)
        self.cnt = np.zeros(part.n_col_blocks, np.int64)
        self.z = {}  # (row block, column block) -> z on the sorted rows of that row block
        self.r = self.y.copy()
        self.rng = S.SplitMix64(self.p["seed"])
        self.epoch = 0
        self.queue = []
        self.drawn_batch = []   # row blocks drawn for the current column batch
        self.drawn_epoch = []   # row blocks drawn in the current epoch
        self.steps = 0
        self.log = []           # per step: dict(j, group, beta, gg, qq, mu)
        self.schedules = []     # the epochs generated so far (for schedule parity)
        self.vb_of_row = [part.row_block_parts(i)[0] for i in range(part.n_row_blocks)]
        self.rows_cache = {}
        self.vox_cache = {}

    # -- helpers --------------------------------------------------------------
    def _rows(self, i):
        if i not in self.rows_cache:
            self.rows_cache[i] = self.part.row_block_rays(i)
        return self.rows_cache[i]

    def _vox(self, j):
        if j not in self.vox_cache:
            self.vox_cache[j] = self.part.tile_voxels(j)
        return self.vox_cache[j]

    def _new_epoch(self):
        ep = S.epoch_schedule(self.rng, self.P, self.p, self.epoch, self.vb_of_row)
        self.schedules.append(ep)
        q = []
        for ci, (j, groups) in enumerate(ep):
            for gi, grp in enumerate(groups):
                q.append((j, grp, gi == len(groups) - 1))
        if not q:
            raise RuntimeError("epoch schedule has no steps (no block can be drawn)")
        self.queue = q

    def _refresh(self, row_blocks):
        """r_It = y_It - sum_j z_It^j over the rows of the given row blocks."""
        for i in sorted(set(row_blocks)):
            rows = self._rows(i)
            acc = np.zeros(rows.shape[0])
            for j in range(self.part.n_col_blocks):
                zz = self.z.get((i, j))
                if zz is not None:
                    acc += zz
            self.r[rows] = self.y[rows] - acc

    def _close_epoch(self):
        if self.p["sync"] == EPOCH:
            self._refresh(self.drawn_epoch)
        elif self.drawn_batch:
            self._refresh(self.drawn_batch)
        for j in range(self.part.n_col_blocks):
            if self.cnt[j] > 0:
                v = self._vox(j)
                self.x[v] = self.xhat[v] / self.cnt[j]
        self.xhat[:] = 0.0
        self.cnt[:] = 0
        self.drawn_batch = []
        self.drawn_epoch = []
        self.queue = []
        self.epoch += 1

    # -- Alg. 1 -------------------------------------------------------------
    def step(self, j: int, group) -> dict:
        part = self.part
        rows = part.rows_of(group)
        vox = self._vox(j)
        g_full = backproject_block(part, group, j, self.r[rows])
        gJ = g_full[vox]
        _, q = project_block(part, group, j, g_full)
        gg = float(np.dot(gJ, gJ))
        qq = float(np.dot(q, q))
        beta = self.p["b"] * float(sum(self.P[i, j] for i in group))
        mu = step_length(beta, gg, qq)
        c = np.zeros_like(self.x)
        c[vox] = self.x[vox] + mu * gJ
        self.xhat[vox] += c[vox]
        self.cnt[j] += 1
        for i in group:
            _, zz = project_block(part, [i], j, c)
            self.z[(i, j)] = zz
        info = dict(j=j, group=list(group), beta=beta, gg=gg, qq=qq, mu=mu)
        self.log.append(info)
        self.steps += 1
        return info

    def run(self, n_steps: int) -> np.ndarray:
        """n steps of Alg. 2/3/4 from the current state; closes the epoch at the end."""
        for _ in range(int(n_steps)):
            if not self.queue:
                self._new_epoch()
            j, grp, last_in_batch = self.queue.pop(0)
            self.step(j, grp)
            self.drawn_batch.extend(grp)
            self.drawn_epoch.extend(grp)
            if last_in_batch:
                if self.p["sync"] == COLUMN:
                    self._refresh(self.drawn_batch)
                self.drawn_batch = []
            if not self.queue:
                self._close_epoch()
        if self.queue or self.drawn_batch or self.drawn_epoch:
            self._close_epoch()
        return self.x.copy()

    def run_epochs(self, n_epochs: int) -> np.ndarray:
        for _ in range(int(n_epochs)):
            self._new_epoch()
            self.run(len(self.queue))  # consumes exactly the epoch just drawn
        return self.x.copy()
