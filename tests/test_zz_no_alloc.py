"""The allocation-free backprojection against the ordinary one (GPU).

``csgd_backproject_block_noalloc`` serves callers that must not allocate device
memory while they run (a real-time loop planned in advance, or a host that
hands out all device memory at start-up).  It keeps its scratch in a fixed
array inside the library, shared by all calls.  This file is named so that
pytest collects it last; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth import configs as C  # noqa: E402


@pytest.fixture(scope="module")
def csgd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_00953_gb300 import build as B
    B.build()
    from paper_1709_00953_gb300 import csgd as M
    return M


def _setup(csgd, cfg):
    g = csgd.Geometry(cfg["geom"])
    p = csgd.Partition(g, **cfg["part"])
    # one ordinary device call uploads the partition's tables
    x = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
    out = torch.zeros(p.n_rays, dtype=torch.float32, device="cuda")
    csgd.project_block(p, [0], 0, x, out)
    return p


@pytest.mark.parametrize("cfg", [C.small_fan2d(n=96, views=48, nu=144, tiles=(3, 3), vb=4, du=2),
                                 C.small_cone3d(n=24, views=12, nd=40, tiles=(2, 2, 3), du=2, dv=2)],
                         ids=["fan2d", "cone3d"])
def test_noalloc_matches_backproject_block_twice(csgd, cfg):
    p = _setup(csgd, cfg)
    rng = np.random.default_rng(7)
    calls = [([0, 2], 1), ([p.m - 1], p.n - 1)]
    for k, (grp, j) in enumerate(calls):  # two calls in a row share the fixed array
        r = torch.tensor(rng.standard_normal(p.n_rays).astype(np.float32), device="cuda")
        ref = torch.full((p.n_voxels,), 0.5, dtype=torch.float32, device="cuda")
        got = ref.clone()
        csgd.backproject_block(p, grp, j, r, ref)
        csgd.backproject_block_noalloc(p, grp, j, r, got)
        torch.cuda.synchronize()
        # the same kernels on the same records in the same order: bit for bit
        assert torch.equal(got, ref), k
        assert bool((got != 0.5).any())
        # accumulate mode adds on top of what is there
        once = torch.zeros_like(got)
        csgd.backproject_block_noalloc(p, grp, j, r, once)
        twice = once.clone()
        csgd.backproject_block_noalloc(p, grp, j, r, twice, accumulate=True)
        # x + x is exact in floating point
        assert torch.equal(twice, 2 * once)


def test_noalloc_rejects_too_many_rays(csgd):
    cfg = C.cone3d_256()
    cfg["geom"]["angles"] = cfg["geom"]["angles"][:4]
    cfg["part"] = dict(tiles=(1, 1, 1), view_blocks=1, det_blocks=(1, 1))
    g = csgd.Geometry(cfg["geom"])
    p = csgd.Partition(g, **cfg["part"])
    x = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
    out = torch.zeros(p.n_rays, dtype=torch.float32, device="cuda")
    csgd.project_block(p, [0], 0, x, out)
    r = torch.zeros(p.n_rays, dtype=torch.float32, device="cuda")
    gv = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
    # 4 views x 384 x 384 bins, all in the single tile's shadow: > 262144 rays
    with pytest.raises(csgd.CsgdError) as e:
        csgd.backproject_block_noalloc(p, [0], 0, r, gv)
    assert e.value.code == -1 and "CSGD_NOALLOC_MAX_RAYS" in str(e.value)


def test_noalloc_needs_tables_on_device(csgd):
    cfg = C.small_fan2d(n=48, views=12, nu=72, tiles=(2, 2), vb=2, du=1)
    g = csgd.Geometry(cfg["geom"])
    p = csgd.Partition(g, **cfg["part"])
    r = torch.zeros(p.n_rays, dtype=torch.float32, device="cuda")
    gv = torch.zeros(p.n_voxels, dtype=torch.float32, device="cuda")
    with pytest.raises(csgd.CsgdError) as e:
        csgd.backproject_block_noalloc(p, [0], 0, r, gv)
    assert e.value.code == -5
