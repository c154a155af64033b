"""Batched solves (one CUDA-graph launch for many problems) against solo solves (GPU).

The batched and the one-by-one paths run the same deterministic kernels on
independent state, so every problem's reconstruction must be identical.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import configs as C  # noqa: E402
from synth import data as D  # noqa: E402


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_00953_gb300 import build as B
    B.build()
    from paper_1709_00953_gb300 import batch, csgd
    return csgd, batch


def _problems(batch, k=6):
    cfgs = C.batch_fan2d(n_problems=k, n_range=(64, 160), views_range=(30, 120), epochs=2,
                         seed=42)
    return [batch.Problem(c, D.make_data(c)[0]) for c in cfgs]


def test_graph_solve_equals_plain_solve(mods):
    csgd, batch = mods
    (p,) = _problems(batch, 1)
    g = p.graph()
    g.launch()
    torch.cuda.synchronize()
    x_graph = p.x.clone()
    p.x.zero_()
    p.solve_plain()
    torch.cuda.synchronize()
    assert torch.equal(p.x, x_graph)
    # a second launch repeats the same solve
    p.x.zero_()
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(p.x, x_graph)


def test_batch_equals_one_by_one(mods):
    csgd, batch = mods
    probs = _problems(batch, 6)
    b = batch.Batch(probs)
    b.launch()
    torch.cuda.synchronize()
    xs = [p.x.clone() for p in probs]
    for p in probs:
        p.x.fill_(-1.0)
    b.solve_one_by_one()
    for p, xb in zip(probs, xs):
        assert torch.equal(p.x, xb), p.cfg["name"]
        assert float(p.x.abs().max()) > 0


def test_graph_to_pinned_host(mods):
    csgd, batch = mods
    (p,) = _problems(batch, 1)
    host = torch.empty(p.partition.n_voxels, dtype=torch.float32).pin_memory()
    g = p.solver.graph(p.steps, host)
    g.launch()
    torch.cuda.synchronize()
    p.solve_plain()
    torch.cuda.synchronize()
    assert torch.equal(host, p.x.cpu())
    with pytest.raises(csgd.CsgdError):
        p.solver.graph(p.steps, torch.empty(p.partition.n_voxels, dtype=torch.float32))


def test_launch_shapes_change_rounding_only(mods):
    """Every launch shape (view groups per backprojection CTA or the scatter, lanes per ray) gives
    the same solve to rounding; autotuning picks a valid shape and resets."""
    csgd, batch = mods
    cfg = C.small_fan2d(n=96, views=48, nu=144, tiles=(3, 3), vb=4, du=2)
    y, _ = D.make_data(cfg)
    p = csgd.Partition(csgd.Geometry(cfg["geom"]), **cfg["part"])
    yt = torch.tensor(y, device="cuda")
    s = csgd.Solver(p, cfg["solver"], yt)
    steps = 24

    def run(c, l):
        s.set_launch(c, l)
        s.reset(yt)
        x = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
        s.solve(steps, x, report=False)
        torch.cuda.synchronize()
        return x.cpu().numpy().astype(np.float64)

    ref = run(0, 0)
    for c in list(range(1, 9)) + [csgd.SCATTER] + list(csgd.BRICKS):
        for l in (1, 2, 4):
            x = run(c, l)
            assert np.sqrt(np.mean((x - ref) ** 2)) <= 1e-5 * max(np.abs(ref).max(), 1e-12), (c, l)
    c, l = s.autotune(8)
    assert (c == csgd.SCATTER or c in csgd.BRICKS or 1 <= c <= 8) and l in (1, 2, 4)
    with pytest.raises(RuntimeError):
        s.set_launch(9, 0)
    with pytest.raises(RuntimeError):
        s.set_launch(min(csgd.BRICKS) - 1, 0)
    with pytest.raises(RuntimeError):
        s.set_launch(0, 3)


def test_batch_matches_oracle(mods):
    """Batched solves against the FP64 oracle: three uneven problems of the
    batched workload's kind (curved fans, 8 view blocks x 4 x 4 tiles,
    density-weighted choice), autotuned and solved together in one graph
    launch, each within RMSE 1e-4 of the oracle's literal run of its own
    schedule and step count."""
    from oracle.blocks import Partition as OPart
    from oracle.geometry import Geometry as OGeom
    from oracle.solver import OracleSolver
    csgd, batch = mods
    probs = _problems(batch, 3)
    b = batch.Batch(probs, autotune=True)
    b.launch()
    torch.cuda.synchronize()
    for p in probs:
        cfg = p.cfg
        og = OGeom(**cfg["geom"])
        op = OPart(og, cfg["part"]["tiles"], cfg["part"]["view_blocks"], cfg["part"]["det_blocks"])
        o = OracleSolver(op, cfg["solver"], p.y.cpu().numpy().astype(np.float64))
        xo = o.run(p.steps)
        xg = p.x.cpu().numpy().astype(np.float64)
        assert np.abs(xo).max() > 0
        assert float(np.sqrt(np.mean((xg - xo) ** 2))) <= 1e-4, cfg["name"]
