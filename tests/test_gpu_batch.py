"""Batched solves against solo solves and the oracle (GPU).

Two batched forms: one persistent launch of the executor with its device work
queue (``Batch.launch``), and a graph of the problems' solve graphs
(``Batch.launch_graphs``).  The graph form runs the same deterministic kernels
on independent state as the one-by-one solves, so it must equal them bit for
bit; the executor runs the same kernel bodies with one lane per ray and
256-thread blocks, so it must equal them to rounding, repeat itself bit for
bit, and match the oracle.  A bounded wait that runs out must end the launch
with CSGD_ERR_TIMEOUT and leave the context usable.
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
    b.launch_graphs()
    torch.cuda.synchronize()
    xs = [p.x.clone() for p in probs]
    for p in probs:
        p.x.fill_(-1.0)
    b.solve_one_by_one()
    for p, xb in zip(probs, xs):
        assert torch.equal(p.x, xb), p.cfg["name"]
        assert float(p.x.abs().max()) > 0
    # the same graphs launched one after the other
    for p in probs:
        p.x.fill_(-1.0)
    b.launch_sequential_graphs()
    torch.cuda.synchronize()
    for p, xb in zip(probs, xs):
        assert torch.equal(p.x, xb), p.cfg["name"]


def test_executor_equals_one_by_one_to_rounding(mods):
    """The persistent launch: every problem's x within rounding of its own
    host-launched solve with the executor's launch shapes (4 view groups, the
    solver's lanes per ray: 1, 2 and 4 here), bit for bit from one launch to
    the next, status OK."""
    csgd, batch = mods
    probs = _problems(batch, 6)
    for k, p in enumerate(probs):
        p.solver.set_launch(4, (1, 2, 4)[k % 3])
    b = batch.Batch(probs)
    info = b.executor.info()
    assert info["tasks"] > 6 and info["units"] > info["tasks"] and info["blocks"] > 0
    b.launch()
    b.status()
    xs = [p.x.clone() for p in probs]
    for p in probs:
        p.x.fill_(-1.0)
    b.launch()
    b.status()
    for p, xe in zip(probs, xs):
        assert torch.equal(p.x, xe), p.cfg["name"]
    b.solve_one_by_one()
    for p, xe in zip(probs, xs):
        ref = p.x.double()
        err = float(torch.sqrt(torch.mean((xe.double() - ref) ** 2)))
        assert err <= 1e-5 * float(ref.abs().max()), (p.cfg["name"], err)


def test_executor_3d_and_scatter(mods):
    """Cone problems through the executor with the scatter backprojection (its
    lines set up inline, max |r| per slot, fixed-point sums): within rounding
    of the solvers' own solves."""
    csgd, batch = mods
    cfgs = [C.small_cone3d(n=20, views=12, nd=32, tiles=(2, 2, 2), group=3, steps=16),
            C.small_cone3d(n=24, views=16, nd=40, tiles=(2, 2, 3), group=4, steps=20)]
    probs = [batch.Problem(c, D.make_data(c)[0]) for c in cfgs]
    for p, lanes in zip(probs, (1, 2)):
        p.solver.set_launch(csgd.SCATTER, lanes)
    b = batch.Batch(probs)
    b.launch()
    b.status()
    xs = [p.x.clone() for p in probs]
    b.solve_one_by_one()
    for p, xe in zip(probs, xs):
        ref = p.x.double()
        err = float(torch.sqrt(torch.mean((xe.double() - ref) ** 2)))
        assert float(ref.abs().max()) > 0
        assert err <= 1e-5 * float(ref.abs().max()), (p.cfg["name"], err)


def test_executor_wait_runs_out(mods):
    """The last task of the first problem waits for a block of work that never
    completes (a test hook): its wait must run out after the limit (0.2 s of
    GPU time), the launch end with CSGD_ERR_TIMEOUT, and the context stay
    usable (a normal batch then runs)."""
    csgd, batch = mods
    probs = _problems(batch, 2)
    stalled = csgd.Batch([p.solver for p in probs], [p.steps for p in probs],
                         [p.x for p in probs], wait_limit_ns=200_000_000, stall_last_task=True)
    stalled.launch()
    with pytest.raises(csgd.CsgdError) as e:
        stalled.status()
    assert e.value.code == -4
    del stalled
    ok = csgd.Batch([p.solver for p in probs], [p.steps for p in probs], [p.x for p in probs])
    ok.launch()
    ok.status()
    assert all(float(p.x.abs().max()) > 0 for p in probs)


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
    density-weighted choice), autotuned and solved together in one persistent
    launch, each within RMSE 1e-4 of the oracle's literal run of its own
    schedule and step count."""
    from oracle.blocks import Partition as OPart
    from oracle.geometry import Geometry as OGeom
    from oracle.solver import OracleSolver
    csgd, batch = mods
    probs = _problems(batch, 3)
    b = batch.Batch(probs, autotune=True)
    b.launch()
    b.status()
    for p in probs:
        cfg = p.cfg
        og = OGeom(**cfg["geom"])
        op = OPart(og, cfg["part"]["tiles"], cfg["part"]["view_blocks"], cfg["part"]["det_blocks"])
        o = OracleSolver(op, cfg["solver"], p.y.cpu().numpy().astype(np.float64))
        xo = o.run(p.steps)
        xg = p.x.cpu().numpy().astype(np.float64)
        assert np.abs(xo).max() > 0
        assert float(np.sqrt(np.mean((xg - xo) ** 2))) <= 1e-4, cfg["name"]
