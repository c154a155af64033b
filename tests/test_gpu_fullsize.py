"""GPU parity at the benchmark's full sizes, on outputs the oracle can compute.

* fan2d_512 (the benchmark workload, same partition, data, parameters and
  kernels as ``bench.py``): the first block step's beta, g^T g, q^T q and mu, the
  tile after that step (a one-step run closes the epoch, so x_J is the step's
  candidate), and sampled rays of the full forward projection A x.
* cone3d_256: sampled rays of one view's block projection, the backprojection of
  one view on one tile, and one grouped step on an explicit small group.

Tolerances are those of ``test_gpu_parity.py``.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import blocks as OB  # noqa: E402
from oracle import siddon as OSd  # noqa: E402
from oracle.blocks import Partition as OPart  # noqa: E402
from oracle.geometry import Geometry as OGeom  # noqa: E402
from oracle.solver import OracleSolver  # noqa: E402
from synth import configs as C  # noqa: E402
from synth import data as D  # noqa: E402

REL = 1e-5
TAU_GEOM = 2.0 ** -14
TAU_BP = 2.0 ** -12


@pytest.fixture(scope="module")
def csgd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_00953_gb300 import build as B
    B.build()
    from paper_1709_00953_gb300 import csgd as M
    return M


def _pair(csgd, cfg):
    p = csgd.Partition(csgd.Geometry(cfg["geom"]), **cfg["part"])
    og = OGeom(**cfg["geom"])
    op = OPart(og, cfg["part"]["tiles"], cfg["part"]["view_blocks"], cfg["part"]["det_blocks"])
    return p, op


@pytest.fixture(scope="module")
def fan(csgd):
    cfg = C.fan2d_512()
    y, _ = D.make_data(cfg)
    p, op = _pair(csgd, cfg)
    return cfg, y, p, op


def test_fan512_first_step_matches_oracle(csgd, fan):
    cfg, y, p, op = fan
    s = csgd.Solver(p, cfg["solver"], torch.tensor(y, device="cuda"))
    x = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
    s.solve(1, x)
    h = s.history()[0]
    o = OracleSolver(op, cfg["solver"], y.astype(np.float64))
    xo = o.run(1)
    ref = o.log[0]
    assert h["beta"] == pytest.approx(ref["beta"], rel=1e-12)
    assert h["gg"] == pytest.approx(ref["gg"], rel=REL)
    assert h["qq"] == pytest.approx(ref["qq"], rel=REL)
    assert h["mu"] == pytest.approx(ref["mu"], rel=REL)
    vox = op.tile_voxels(ref["j"])
    xg = x.cpu().numpy().astype(np.float64)
    assert np.all(np.delete(xg, vox) == 0.0)
    err = np.abs(xg[vox] - xo[vox])
    assert err.max() <= REL * np.abs(xo[vox]).max() + 1e-7, err.max()
    # non-zeros visited by the step = nnz(A_{I_g}^J) counted by the oracle
    assert h["nnz"] == pytest.approx(OB.block_nnz(op, ref["group"], ref["j"]), rel=1e-4)


def test_fan512_full_forward_sampled_rays(csgd, fan):
    cfg, y, p, op = fan
    rng = np.random.default_rng(3)
    x = rng.random(p.n_voxels).astype(np.float32)
    out = torch.zeros(p.n_rays, dtype=torch.float32, device="cuda")
    csgd.project_full(p, torch.tensor(x, device="cuda"), out)
    rays = rng.choice(p.n_rays, 3000, replace=False)
    g = op.geom
    o, d = g.rays(rays)
    ref = OSd.project_box(g.grid, o, d, [0, 0], list(g.n), x.astype(np.float64))
    got = out.cpu().numpy()[rays].astype(np.float64)
    tol = REL * ref + TAU_GEOM * np.abs(x).max() * op.n_col_blocks
    assert np.all(np.abs(got - ref) <= tol)


@pytest.fixture(scope="module")
def cone(csgd):
    cfg = C.cone3d_256()
    p, op = _pair(csgd, cfg)
    return cfg, p, op


def test_cone256_project_block_sampled_rays(csgd, cone):
    cfg, p, op = cone
    rng = np.random.default_rng(4)
    x = rng.random(p.n_voxels).astype(np.float32)
    xt = torch.tensor(x, device="cuda")
    for view, j in ((0, 21), (97, 42), (250, 0)):
        out = torch.zeros(p.n_rays, dtype=torch.float32, device="cuda")
        csgd.project_block(p, [view], j, xt, out)
        rows = op.row_block_rays(view)
        pick = rng.choice(rows, 2000, replace=False)
        g = op.geom
        o, d = g.rays(pick)
        lo, hi = op.tile_box(j)
        ref = OSd.project_box(g.grid, o, d, lo, hi, x.astype(np.float64))
        got = out.cpu().numpy()[pick].astype(np.float64)
        tol = REL * ref + TAU_GEOM * x.max()
        assert np.all(np.abs(got - ref) <= tol), (view, j)
        assert ref.max() > 0


def test_cone256_backproject_one_view(csgd, cone):
    cfg, p, op = cone
    rng = np.random.default_rng(5)
    r = rng.standard_normal(p.n_rays).astype(np.float32)
    rt = torch.tensor(r, device="cuda")
    view, j = 33, 26
    gv = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
    csgd.backproject_block(p, [view], j, rt, gv)
    rows = op.rows_of([view])
    ref = OB.backproject_block(op, [view], j, r[rows].astype(np.float64))
    absref = OSd.backproject_box(op.geom.grid, *op.geom.rays(rows), *op.tile_box(j),
                                 np.abs(r[rows]).astype(np.float64))
    vox = op.tile_voxels(j)
    got = gv.cpu().numpy().astype(np.float64)[vox]
    tol = REL * absref[vox] + TAU_BP * np.abs(r).max()
    assert np.all(np.abs(got - ref[vox]) <= tol)
    assert np.abs(ref[vox]).max() > 0


def test_cone256_grouped_step(csgd, cone):
    cfg, p, op = cone
    y, _ = D.make_data(cfg, device="cuda")
    s = csgd.Solver(p, cfg["solver"], torch.tensor(y, device="cuda"))
    grp, j = [10, 11, 190], 37
    info = s.step(j=j, row_blocks=grp)
    o = OracleSolver(op, cfg["solver"], y.astype(np.float64))
    ref = o.step(j, grp)
    assert info["beta"] == pytest.approx(ref["beta"], rel=1e-12)
    assert info["gg"] == pytest.approx(ref["gg"], rel=REL)
    assert info["qq"] == pytest.approx(ref["qq"], rel=REL)
    assert info["mu"] == pytest.approx(ref["mu"], rel=REL)
