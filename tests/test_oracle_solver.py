"""Pins of the oracle's Alg. 1-4 (Sec. II-B .. II-E) and the Sec. III measures."""
import numpy as np
import pytest

from oracle import metrics, siddon
from oracle import schedule as S
from oracle.blocks import Partition, backproject_block, project_block
from oracle.geometry import Geometry, uniform_angles
from oracle.solver import COLUMN, EPOCH, OracleSolver


def _tiny(nviews=24, n=6, tiles=(1, 1), vb=1, du=1, nu=10):
    g = Geometry("parallel2d", (n, n), 1.0, uniform_angles(nviews, 180), nu=nu, pu=0.8)
    return Partition(g, tiles=tiles, view_blocks=vb, det_blocks=(du, 1))


def test_single_step_decrease_identity():
    """Eq. 'step' with r^T q = g^T g gives ||r_I||^2 - ||r_I - mu q||^2 = (2 beta - beta^2) gg^2/qq."""
    part = _tiny(12, 8, tiles=(2, 2), vb=3, du=2)
    rng = np.random.default_rng(0)
    y = rng.random(part.geom.n_rays) * 5
    for beta in (0.3, 1.0, 1.7):
        grp, j = [1, 4], 2
        rows = part.rows_of(grp)
        r = y[rows]
        g = backproject_block(part, grp, j, r)
        _, q = project_block(part, grp, j, g)
        gJ = g[part.tile_voxels(j)]
        gg, qq = gJ @ gJ, q @ q
        assert abs(r @ q - gg) <= 1e-12 * gg
        mu = beta * gg / qq
        lhs = r @ r - (r - mu * q) @ (r - mu * q)
        rhs = (2 * beta - beta * beta) * gg * gg / qq
        assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


def test_steepest_descent_reaches_least_squares():
    """m = n = 1 and beta = 1: CSGD is steepest descent with exact line search on
    ||y - Ax||^2, so it converges to the least-squares solution."""
    g = Geometry("parallel2d", (4, 4), 1.0, uniform_angles(40, 180), nu=16, pu=0.3)
    part = Partition(g, tiles=(1, 1))
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d).toarray()
    assert np.linalg.matrix_rank(A) == A.shape[1]
    rng = np.random.default_rng(1)
    y = A @ rng.random(A.shape[1]) + 0.05 * rng.standard_normal(A.shape[0])
    x_ls = np.linalg.lstsq(A, y, rcond=None)[0]
    sol = OracleSolver(part, dict(sampling=S.SEQUENTIAL, b=1.0, alpha=1, gamma=1), y)
    assert sol.P[0, 0] == pytest.approx(1.0)
    x = sol.run(400)  # condition number 3.3: the error shrinks ~4x per 10 steps
    assert np.max(np.abs(x - x_ls)) < 1e-8


def test_column_action_residual_is_exact_and_monotone():
    """m = 1: after every epoch r = y - A x exactly, and ||r|| never grows for 0 < beta < 2."""
    part = _tiny(20, 8, tiles=(2, 2), nu=12)
    g = part.geom
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d)
    y = np.random.default_rng(2).random(g.n_rays) * 3
    sol = OracleSolver(part, dict(sampling=S.UNIFORM, b=1.4, seed=9), y)
    last = np.linalg.norm(y)
    for ep in range(6):
        x = sol.run_epochs(1)
        res = y - A @ x
        np.testing.assert_allclose(sol.r, res, rtol=0, atol=1e-12)
        assert np.linalg.norm(res) <= last * (1 + 1e-14)
        last = np.linalg.norm(res)


def test_epoch_average_of_candidates():
    """m = 2 row blocks, one tile: x_J after the epoch is the mean of the two candidates
    x_J + mu_i g_i, and both steps of the column batch read the batch-start residual
    r = y (Alg. 2)."""
    part = _tiny(16, 6, vb=2, nu=9)
    y = np.random.default_rng(3).random(part.geom.n_rays)
    sol = OracleSolver(part, dict(sampling=S.SEQUENTIAL, b=2.0), y)
    x = sol.run_epochs(1)
    cands = []
    for i in range(2):
        rows = part.rows_of([i])
        gfull = backproject_block(part, [i], 0, y[rows])
        _, q = project_block(part, [i], 0, gfull)
        gJ = gfull[part.tile_voxels(0)]
        beta = 2.0 * sol.P[i, 0]
        cands.append(beta * (gJ @ gJ) / (q @ q) * gJ)
    np.testing.assert_allclose(x[part.tile_voxels(0)], 0.5 * (cands[0] + cands[1]), rtol=1e-12)
    # and the stored z of each block is A_I^J of its own candidate
    for i in range(2):
        c = np.zeros(part.geom.grid.size)
        c[part.tile_voxels(0)] = cands[i]
        np.testing.assert_allclose(sol.z[(i, 0)], project_block(part, [i], 0, c)[1], rtol=1e-12)


def test_stop_mid_epoch_closes_it():
    part = _tiny(16, 8, tiles=(2, 1), vb=2, nu=12)
    y = np.random.default_rng(4).random(part.geom.n_rays)
    sol = OracleSolver(part, dict(sampling=S.UNIFORM, b=2.0, seed=3), y)
    sol.run(3)  # 4 steps per epoch: stops after the first step of the second batch
    assert sol.epoch == 1 and not sol.queue and sol.cnt.sum() == 0
    # the residual is y - sum of the stored z, on every row
    acc = np.zeros(part.geom.n_rays)
    for (i, j), zz in sol.z.items():
        acc[part.row_block_rays(i)] += zz
    np.testing.assert_allclose(sol.r, y - acc, atol=1e-12)


def test_epoch_sync_reads_epoch_start_residual():
    part = _tiny(16, 8, tiles=(2, 1), vb=1, nu=12)
    y = np.random.default_rng(5).random(part.geom.n_rays)
    sol = OracleSolver(part, dict(sampling=S.SEQUENTIAL, b=1.0, sync=EPOCH), y)
    sol.run(1)
    # both column batches of the first epoch read r = y: the second step's g equals the
    # backprojection of y on tile 1
    sol2 = OracleSolver(part, dict(sampling=S.SEQUENTIAL, b=1.0, sync=EPOCH), y)
    sol2.run_epochs(1)
    g1 = backproject_block(part, [0], 1, y)[part.tile_voxels(1)]
    assert sol2.log[1]["gg"] == pytest.approx(float(g1 @ g1), rel=1e-12)


def test_metrics_closed_forms():
    xt = np.array([3.0, 4.0])
    assert metrics.snr_db(xt, 0.9 * xt) == pytest.approx(20.0)
    assert metrics.rmse([1, 2, 3], [1, 2, 5]) == pytest.approx(np.sqrt(4 / 3))


def test_observation_gap_closed_forms():
    """Sec. III's observation gap 20 log10(||y|| / ||y - A x||) on a 2 x 2 image
    seen by two horizontal parallel rays through the pixel rows (view angle 0,
    bins at +-1/2): A x = (x00 + x10, x01 + x11) with unit lengths.  x = (1, 2,
    3, 4) gives A x = (3, 7); y = (4, 7) leaves the residual (1, 0), so the gap
    is 20 log10(sqrt(65)) = 10 log10(65).  Consistent data y = A x gives an
    infinite gap, and x = 0 gives 0 dB."""
    g = Geometry("parallel2d", (2, 2), 1.0, np.array([0.0]), nu=2, pu=1.0)
    x = np.array([1.0, 2.0, 3.0, 4.0])
    np.testing.assert_allclose(metrics.forward_full(g, x), [3.0, 7.0], rtol=0, atol=1e-14)
    assert metrics.observation_gap_db(g, [4.0, 7.0], x) == pytest.approx(10 * np.log10(65.0),
                                                                          rel=1e-14)
    with np.errstate(divide="ignore"):
        assert metrics.observation_gap_db(g, [3.0, 7.0], x) == np.inf
    assert metrics.observation_gap_db(g, [4.0, 7.0], np.zeros(4)) == pytest.approx(0.0, abs=1e-12)


def test_step_length_one_entry_block():
    """Eq. 'step' on a one-entry block A = [l]: g = l r and q = A g = l^2 r, so
    mu = beta / l^2 for every l > 0, however small (no floor on the gain), and
    with beta = 1 the step solves the row exactly.  A g = 0 takes no step."""
    from oracle.solver import step_length
    r, beta = 3.0, 0.7
    for ln in (0.8, 0.01, 1e-3, 1e-5, 1e-9):
        g = ln * r
        q = ln * g
        assert step_length(beta, g * g, q * q) == pytest.approx(beta / ln ** 2, rel=1e-14)
        assert r - step_length(1.0, g * g, q * q) * q == pytest.approx(0.0, abs=1e-12 * r)
    assert step_length(beta, 0.0, 0.0) == 0.0
    assert step_length(beta, 1.0, 0.0) == 0.0


def test_line_through_tile_corner_has_no_support():
    """A line through a corner of a tile meets it in a point: the block it
    forms with a detector sub-area that sees the tile only there has A_I^J = 0
    exactly (no structural sliver from rounding), so g = 0, q = 0 and mu = 0.
    Odd detector (bin 4 of 9 on the central ray) through the grid centre, which
    is a corner of all four tiles, at view angles that are not multiples of 90
    degrees."""
    from oracle.geometry import Geometry, uniform_angles
    g = Geometry("fan2d_flat", (8, 8), 1.0, uniform_angles(36, 360), nu=9, pu=1.0, sod=20.0,
                 sdd=40.0)
    part = Partition(g, tiles=(2, 2), view_blocks=36, det_blocks=(9, 1))
    for v in (1, 5, 13, 22, 31):
        i = v * 9 + 4  # view v, sub-area = bin 4 alone
        for j in range(4):
            rows, z = project_block(part, [i], j, np.ones(g.grid.size))
            if np.any(z > 0):
                assert z.max() > 1.0  # the line crosses this tile's interior
            else:
                gvec = backproject_block(part, [i], j, np.ones(rows.size))
                assert not np.any(gvec)
        # the central line crosses exactly two of the four tiles' interiors
        crossed = [j for j in range(4)
                   if np.any(project_block(part, [i], j, np.ones(g.grid.size))[1] > 0)]
        assert len(crossed) == 2, (v, crossed)


def _split_cone():
    """A cone scan whose volume is split at the source's plane into two tiles and
    whose detector is split at the same height: a line that reaches the upper
    half of the detector never enters the lower tile (it leaves the source's
    plane upward and stays above it), so A is block diagonal in (I, J) and P
    has exact zeros off the diagonal blocks."""
    g = Geometry("cone3d", (4, 4, 2), 1.0, uniform_angles(16, 360), nu=8, nv=8, pu=1.0, pv=1.0,
                 sod=12.0, sdd=24.0)
    part = Partition(g, tiles=(1, 1, 2), view_blocks=4, det_blocks=(1, 2))
    org, d = g.rays()
    A = siddon.system_matrix(g.grid, org, d).toarray()
    assert np.linalg.matrix_rank(A) == A.shape[1]
    return part, A


@pytest.mark.parametrize("sampling,b,epochs,tol", [(S.IMPORTANCE, 1.0, 300, 1e-8),
                                                   (S.UNIFORM, 2.0, 300, 1e-4)])
def test_many_blocks_reach_the_exact_solution(sampling, b, epochs, tol):
    """m = 8 row blocks (4 view groups x 2 detector halves), n = 2 tiles, the
    column batches, z store, residual refresh and candidate averages of Alg. 3
    over many epochs: on consistent data y = A x* with A of full column rank,
    every step's direction lies in the block's row space and the fixed point
    has r = 0, so the run must reach x*.  Uniform sampling also draws the
    zero-overlap blocks (their candidates x_J count in the mean)."""
    from oracle.ptable import probability_table
    part, A = _split_cone()
    P = probability_table(part)
    for i in range(P.shape[0]):
        upper = part.row_block_parts(i)[1] == 1  # row block i reads the upper half
        assert P[i, 0 if upper else 1] == 0.0 and P[i, 1 if upper else 0] > 0.2
    x_star = np.random.default_rng(3).random(A.shape[1])
    sol = OracleSolver(part, dict(sampling=sampling, alpha=1.0, b=b, seed=5), A @ x_star)
    x = sol.run_epochs(epochs)
    assert np.max(np.abs(x - x_star)) < tol
