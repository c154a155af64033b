"""Serving: jobs arriving over time, continuously batched, against solo solves (GPU).

Each job's result must be identical when it runs alone and when it runs in the
mix; the HBM budget must bound how many jobs run at once.
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
    from paper_1709_00953_gb300 import csgd, serve
    return csgd, serve


def _jobs(serve, n=8, rate_per_s=200.0):
    cfgs = C.serving_jobs(n_jobs=n, seed=77, small=True)
    arrivals = serve.poisson_arrivals(n, rate_per_s=rate_per_s, seed=5)
    return [serve.Job(c, D.make_data(c)[0], float(a), c["name"]) for c, a in zip(cfgs, arrivals)]


def _solo(csgd, job):
    g = csgd.Geometry(job.cfg["geom"])
    p = csgd.Partition(g, **job.cfg["part"])
    s = csgd.Solver(p, job.cfg["solver"], torch.tensor(job.y, device="cuda"))
    x = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
    s.solve(job.cfg["steps"], x, report=False)
    torch.cuda.synchronize()
    return x.cpu().numpy()


def test_served_results_equal_solo_results(mods):
    csgd, serve = mods
    # arrivals ~10 us apart: every small job takes longer than that, so jobs
    # overlap whatever the speed of the kernels
    jobs = _jobs(serve, rate_per_s=1e5)
    srv = serve.Server(hbm_budget_bytes=8 << 30, max_running=8)
    srv.run(jobs)
    assert srv.max_concurrency >= 2  # jobs did overlap
    for j in jobs:
        assert j.done > 0 and j.latency > 0
        np.testing.assert_array_equal(j.x, _solo(csgd, j), err_msg=j.name)
    s = serve.summary(jobs, max(j.done for j in jobs))
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_budget_bounds_concurrency(mods):
    csgd, serve = mods
    jobs = _jobs(serve, 5)
    biggest = max(serve.job_footprint(j.cfg) for j in jobs)
    srv = serve.Server(hbm_budget_bytes=biggest, max_running=8)
    for j in jobs:
        j.arrival = 0.0
    srv.run(jobs)
    # admission never lets the running jobs' footprints exceed the budget
    assert 0 < srv.max_used <= biggest
    assert srv.max_concurrency < len(jobs)
    for j in jobs:
        assert j.x is not None
    too_small = serve.Server(hbm_budget_bytes=biggest // 4, max_running=2)
    with pytest.raises(ValueError):
        too_small.run(_jobs(serve, 5))


def test_served_results_match_the_oracle(mods):
    """Served reconstructions against the FP64 oracle's solution of the same job
    (same data, schedule and step count): RMSE <= 1e-3, the serving quality bar."""
    from oracle.blocks import Partition as OPart
    from oracle.geometry import Geometry as OGeom
    from oracle.solver import OracleSolver
    csgd, serve = mods
    mix = _jobs(serve)
    jobs = [next(j for j in mix if "cone3d" in j.name), next(j for j in mix if "fan2d" in j.name)]
    srv = serve.Server(hbm_budget_bytes=8 << 30, max_running=8)
    srv.run(jobs)
    for j in jobs:
        cfg = j.cfg
        og = OGeom(**cfg["geom"])
        op = OPart(og, cfg["part"]["tiles"], cfg["part"]["view_blocks"], cfg["part"]["det_blocks"])
        xo = OracleSolver(op, cfg["solver"], j.y.astype(np.float64)).run(cfg["steps"])
        rmse = float(np.sqrt(np.mean((j.x.astype(np.float64) - xo) ** 2)))
        assert rmse <= 1e-3, (j.name, rmse)
