"""Pins of the oracle's block structure (Eq. e1): reassembly and adjoint identity."""
import numpy as np
import pytest

from oracle import siddon
from oracle.blocks import Partition, backproject_block, block_matrix, project_block
from oracle.geometry import Geometry, uniform_angles


def _cases():
    return [
        Partition(Geometry("parallel2d", (10, 9), 1.0, uniform_angles(7, 180), nu=14, pu=1.0),
                  tiles=(3, 2), view_blocks=3, det_blocks=(2, 1)),
        Partition(Geometry("fan2d_curved", (12, 12), 1.0, uniform_angles(9, 360), nu=20,
                           pu=0.06, sod=24, sdd=48), tiles=(2, 3), view_blocks=2, det_blocks=(3, 1)),
        Partition(Geometry("cone3d", (6, 7, 5), 1.0, uniform_angles(5, 360), nu=9, nv=8,
                           pu=2.0, pv=2.0, sod=15, sdd=30), tiles=(2, 2, 2), view_blocks=5,
                  det_blocks=(2, 2)),
    ]


@pytest.mark.parametrize("k", range(3))
def test_reassembly(k):
    """sum over (I, J) of embed(A_I^J) = A: every non-zero lies in exactly one block."""
    part = _cases()[k]
    g = part.geom
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d).toarray()
    R = np.zeros_like(A)
    hits = np.zeros_like(A, dtype=np.int64)
    for i in range(part.n_row_blocks):
        rows = part.rows_of([i])
        for j in range(part.n_col_blocks):
            B = block_matrix(part, [i], j).toarray()
            cols = part.tile_voxels(j)
            R[np.ix_(rows, cols)] += B
            hits[np.ix_(rows, cols)] += 1
    np.testing.assert_allclose(R, A, rtol=1e-12, atol=0)
    assert np.all(hits == 1)  # the blocks tile the index space exactly once
    assert part.rows_of(range(part.n_row_blocks)).shape[0] == g.n_rays


@pytest.mark.parametrize("k", range(3))
def test_block_operators_and_adjoint(k):
    part = _cases()[k]
    g = part.geom
    rng = np.random.default_rng(k)
    x = rng.standard_normal(g.grid.size)
    for grp in ([0], [0, part.n_row_blocks - 1]):
        for j in (0, part.n_col_blocks - 1):
            rows, p = project_block(part, grp, j, x)
            B = block_matrix(part, grp, j)
            vox = part.tile_voxels(j)
            np.testing.assert_allclose(p, B @ x[vox], rtol=1e-12, atol=1e-12)
            r = rng.standard_normal(rows.shape[0])
            gfull = backproject_block(part, grp, j, r)
            assert np.all(np.delete(gfull, vox) == 0.0)
            np.testing.assert_allclose(gfull[vox], B.T @ r, rtol=1e-12, atol=1e-12)
            lhs = float(np.dot(p, r))
            rhs = float(np.dot(x[vox], gfull[vox]))
            assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_ragged_tiles_cover_grid():
    part = Partition(Geometry("parallel2d", (64, 61), 1.0, uniform_angles(4, 180), nu=90),
                     tiles=(3, 5))
    seen = np.zeros(64 * 61, np.int64)
    for j in range(part.n_col_blocks):
        seen[part.tile_voxels(j)] += 1
    assert np.all(seen == 1)
    assert part.tile_box(0) == ([0, 0], [21, 12])
    assert part.tile_box(part.n_col_blocks - 1) == ([42, 48], [64, 61])
