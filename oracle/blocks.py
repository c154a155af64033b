"""Row blocks I, column blocks J and the block operators (Eq. e1, Sec. II-D), FP64.

Test infrastructure only (see the package docstring).

Eq. (e1) splits the rows and columns of A into index sets I_1..I_m and
J_1..J_n; Sec. II-D builds them for tomography from cuboid volume tiles and,
per view, detector sub-areas.  The readings used throughout:

* column block (tile) j = (tz * TY + ty) * TX + tx; along an axis with N voxels
  and T tiles, tile t covers voxels [floor(t N / T), floor((t+1) N / T));
* row block i = (vb * DV + dv) * DU + du: a set of views (view block vb,
  either contiguous views split at floor(k V / VB) or an explicit view -> block
  map) times a detector sub-rectangle (u-bins split at floor(k nu / DU), v-bins
  split at floor(k nv / DV));
* A_I^J is A restricted to rows in I and columns in J, nothing else.

Parity: pinned by reassembly (every non-zero of A in exactly one block) and by
the adjoint identity in ``tests/test_oracle_blocks.py``.
"""
from __future__ import annotations

import numpy as np

from . import siddon
from .geometry import Geometry


def _splits(n: int, parts: int) -> np.ndarray:
    return np.array([(k * n) // parts for k in range(parts + 1)], np.int64)


class Partition:
    """The partition of Eq. (e1) for one geometry."""

    def __init__(self, geom: Geometry, tiles, view_blocks: int = 1, det_blocks=(1, 1),
                 view_block_of=None):
        self.geom = geom
        tiles = tuple(int(t) for t in tiles)
        assert len(tiles) == geom.dim
        self.tiles = tiles
        self.tile_edges = [_splits(geom.n[a], tiles[a]) for a in range(geom.dim)]
        du, dv = (tuple(det_blocks) + (1,))[:2]
        self.du, self.dv = int(du), int(dv)
        self.u_edges = _splits(geom.nu, self.du)
        self.v_edges = _splits(geom.nv, self.dv)
        V = geom.n_views
        if view_block_of is None:
            self.vb_count = int(view_blocks)
            e = _splits(V, self.vb_count)
            vbo = np.zeros(V, np.int64)
            for b in range(self.vb_count):
                vbo[e[b]:e[b + 1]] = b
        else:
            vbo = np.asarray(view_block_of, np.int64).reshape(V)
            self.vb_count = int(vbo.max()) + 1
        self.view_block_of = vbo
        self.views_of_vb = [np.nonzero(vbo == b)[0] for b in range(self.vb_count)]

    # ---- sizes -------------------------------------------------------------
    @property
    def n_col_blocks(self) -> int:
        return int(np.prod(self.tiles))

    @property
    def n_row_blocks(self) -> int:
        return self.vb_count * self.dv * self.du

    # ---- column blocks -----------------------------------------------------
    def tile_coords(self, j: int):
        tx = self.tiles[0]
        ty = self.tiles[1]
        c = [j % tx, (j // tx) % ty]
        if self.geom.dim == 3:
            c.append(j // (tx * ty))
        return c

    def tile_box(self, j: int):
        """Index box [lo, hi) of tile j, one entry per axis (x first)."""
        c = self.tile_coords(j)
        lo = [int(self.tile_edges[a][c[a]]) for a in range(self.geom.dim)]
        hi = [int(self.tile_edges[a][c[a] + 1]) for a in range(self.geom.dim)]
        return lo, hi

    def tile_voxels(self, j: int) -> np.ndarray:
        """Sorted linear indices of the voxels in tile j (the set J_j)."""
        lo, hi = self.tile_box(j)
        n = self.geom.n
        ax = [np.arange(lo[a], hi[a]) for a in range(self.geom.dim)]
        if self.geom.dim == 2:
            yy, xx = np.meshgrid(ax[1], ax[0], indexing="ij")
            return (yy * n[0] + xx).reshape(-1)
        zz, yy, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return ((zz * n[1] + yy) * n[0] + xx).reshape(-1)

    # ---- row blocks --------------------------------------------------------
    def row_block_parts(self, i: int):
        du = i % self.du
        dv = (i // self.du) % self.dv
        vb = i // (self.du * self.dv)
        return vb, dv, du

    def row_block_subrect(self, i: int):
        """(u0, u1, v0, v1): the detector sub-rectangle of row block i."""
        vb, dv, du = self.row_block_parts(i)
        return (int(self.u_edges[du]), int(self.u_edges[du + 1]),
                int(self.v_edges[dv]), int(self.v_edges[dv + 1]))

    def row_block_views(self, i: int) -> np.ndarray:
        vb, _, _ = self.row_block_parts(i)
        return self.views_of_vb[vb]

    def row_block_rays(self, i: int) -> np.ndarray:
        """Sorted global indices of the measurements in row block i (the set I_i)."""
        u0, u1, v0, v1 = self.row_block_subrect(i)
        g = self.geom
        kv, ku = np.meshgrid(np.arange(v0, v1), np.arange(u0, u1), indexing="ij")
        within = (kv * g.nu + ku).reshape(-1)
        views = self.row_block_views(i)
        return (views[:, None] * g.rays_per_view + within[None, :]).reshape(-1)

    def rows_of(self, row_blocks) -> np.ndarray:
        """Sorted union of the rows of several row blocks (I_g of Alg. 4)."""
        parts = [self.row_block_rays(int(i)) for i in row_blocks]
        if not parts:
            return np.zeros(0, np.int64)
        return np.unique(np.concatenate(parts))


# ---- operators -------------------------------------------------------------
def project_block(part: Partition, row_blocks, j: int, x: np.ndarray):
    """z_I = A_I^J x_J (Alg. 1, last line; Eq. e1), FP64.

    Returns (rows, values): the sorted rows of the union of ``row_blocks`` and
    the restricted forward projection of the tile ``j`` part of the full volume x.
    """
    g = part.geom
    rows = part.rows_of(row_blocks)
    org, d = g.rays(rows)
    lo, hi = part.tile_box(j)
    return rows, siddon.project_box(g.grid, org, d, lo, hi, x)


def backproject_block(part: Partition, row_blocks, j: int, r_rows: np.ndarray):
    """g_J = (A_I^J)^T r_I (Eq. 'direction', Alg. 1), FP64.

    ``r_rows`` holds r on the sorted rows of the union of ``row_blocks``.
    Returns a full-size volume that is zero outside tile j.
    """
    g = part.geom
    rows = part.rows_of(row_blocks)
    r_rows = np.asarray(r_rows, np.float64).reshape(-1)
    assert r_rows.shape[0] == rows.shape[0]
    org, d = g.rays(rows)
    lo, hi = part.tile_box(j)
    return siddon.backproject_box(g.grid, org, d, lo, hi, r_rows)


def block_matrix(part: Partition, row_blocks, j: int):
    """A_I^J as a CSR matrix with rows = rows_of(row_blocks), columns = tile_voxels(j)."""
    g = part.geom
    rows = part.rows_of(row_blocks)
    org, d = g.rays(rows)
    A = siddon.system_matrix(g.grid, org, d)
    return A[:, part.tile_voxels(j)]


def block_nnz(part: Partition, row_blocks, j: int) -> int:
    """Number of non-zeros of A_I^J (I = union of row_blocks, J = tile j)."""
    g = part.geom
    rows = part.rows_of(row_blocks)
    org, d = g.rays(rows)
    lo, hi = part.tile_box(j)
    return siddon.count_box(g.grid, org, d, lo, hi)
