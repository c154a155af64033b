"""Host logic of the C ABI (no GPU needed): symbols, importance table, schedule.

The library's P(I,J) and its block schedule are host FP64 / integer code; they
are compared here with the oracle's independent implementations.
"""
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import ptable as OP
from oracle import schedule as OS
from oracle.blocks import Partition as OPart
from oracle.geometry import Geometry as OGeom
from synth import configs as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_00953_gb300 import build as B
    B.build()
    from paper_1709_00953_gb300 import csgd
    return csgd


def test_library_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "csgd.h")).read()
    declared = set(re.findall(r"^(?:int32_t|const char\*)\s+(csgd_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (csgd_\w+)", out))
    assert declared <= exported, declared - exported
    assert declared == set(lib.SIGNATURES), set(lib.SIGNATURES) ^ declared
    L = lib.load()
    for name in declared:
        assert hasattr(L, name)
    assert "sm_103a" in lib.version()


def _pair(cfg):
    from paper_1709_00953_gb300 import csgd
    g = csgd.Geometry(cfg["geom"])
    p = csgd.Partition(g, **cfg["part"])
    og = OGeom(**cfg["geom"])
    op = OPart(og, cfg["part"]["tiles"], cfg["part"]["view_blocks"], cfg["part"]["det_blocks"])
    return p, op


CASES = [
    C.parallel2d_64(),
    C.small_fan2d(n=64, views=40, nu=96, tiles=(3, 2), vb=4, du=3),
    C.small_fan2d(n=64, views=36, nu=90, tiles=(2, 3), vb=3, du=2, curved=False),
    C.small_cone3d(n=16, views=12, nd=24, tiles=(2, 2, 3), du=2, dv=2),
]


@pytest.mark.parametrize("k", range(len(CASES)))
def test_probability_table_matches_oracle(lib, k):
    p, op = _pair(CASES[k])
    P = p.probabilities()
    Po = OP.probability_table(op)
    assert P.shape == Po.shape
    np.testing.assert_allclose(P, Po, rtol=1e-12, atol=1e-14)


def test_probability_table_cone_full_size(lib):
    cfg = C.cone3d_256()
    cfg["geom"]["angles"] = cfg["geom"]["angles"][::30]
    cfg["part"]["view_blocks"] = 12
    p, op = _pair(cfg)
    np.testing.assert_allclose(p.probabilities(), OP.probability_table(op), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("sampling", [OS.SEQUENTIAL, OS.UNIFORM, OS.IMPORTANCE, OS.MIXED])
@pytest.mark.parametrize("k", [0, 1, 3])
def test_schedule_matches_oracle(lib, k, sampling):
    cfg = CASES[k]
    p, op = _pair(cfg)
    prm = dict(cfg["solver"], sampling=sampling, alpha=0.6, gamma=0.8, group_size=2, seed=77 + k,
               theta_step=0.1)
    flat = lib.schedule_generate(p, prm, 6)
    rng = OS.SplitMix64(prm["seed"])
    P = OP.probability_table(op)
    vb = [op.row_block_parts(i)[0] for i in range(op.n_row_blocks)]
    eps = [OS.epoch_schedule(rng, P, prm, e, vb) for e in range(6)]
    assert flat == OS.flatten(eps)


def test_fan512_schedule_matches_oracle(lib):
    cfg = C.fan2d_512()
    p, op = _pair(cfg)
    flat = lib.schedule_generate(p, cfg["solver"], 4)
    rng = OS.SplitMix64(cfg["solver"]["seed"])
    P = OP.probability_table(op)
    vb = [op.row_block_parts(i)[0] for i in range(op.n_row_blocks)]
    eps = [OS.epoch_schedule(rng, P, cfg["solver"], e, vb) for e in range(4)]
    assert flat == OS.flatten(eps)
    # 16 columns, each with ceil(0.5 * 8) = 4 single-block groups
    assert flat[0] == 16


def test_invalid_arguments_are_rejected(lib):
    from paper_1709_00953_gb300 import csgd
    bad = dict(C.parallel2d_64()["geom"], nu=0)
    with pytest.raises(csgd.CsgdError) as e:
        csgd.Geometry(bad)
    assert e.value.code == -1
    g = csgd.Geometry(C.parallel2d_64()["geom"])
    with pytest.raises(csgd.CsgdError):
        csgd.Partition(g, tiles=(65, 1))
    p = csgd.Partition(g, tiles=(2, 2), view_blocks=2)
    with pytest.raises(csgd.CsgdError):
        csgd.schedule_generate(p, dict(C.parallel2d_64()["solver"], alpha=1.5), 1)
    bad_fan = dict(C.small_fan2d()["geom"], sod=10.0)
    with pytest.raises(csgd.CsgdError):
        csgd.Geometry(bad_fan)
    # 1291^3 voxels (8.6 GB of FP32) is more than 32-bit voxel indices reach
    big = dict(C.cone3d_256()["geom"], n=(1291, 1291, 1291), sod=4000.0, sdd=8000.0)
    with pytest.raises(csgd.CsgdError) as e:
        csgd.Geometry(big)
    assert e.value.code == -1 and "voxels" in str(e.value)
    ok = dict(C.cone3d_256()["geom"], n=(1290, 1290, 1290), sod=4000.0, sdd=8000.0)
    csgd.Geometry(ok)  # 2,146,689,000 < 2^31


def test_footprint_grows_with_problem(lib):
    from paper_1709_00953_gb300 import csgd
    a = C.parallel2d_64()
    b = C.fan2d_512()
    pa = csgd.Partition(csgd.Geometry(a["geom"]), **a["part"])
    pb = csgd.Partition(csgd.Geometry(b["geom"]), **b["part"])
    fa = csgd.footprint_bytes(pa, a["solver"])
    fb = csgd.footprint_bytes(pb, b["solver"])
    assert 0 < fa < fb
    # at least x, xhat, y, r, p, q and the z store
    assert fb >= 4 * (2 * pb.n_voxels + 4 * pb.n_rays + pb.z_floats)


def test_sec3_study_step_counts(lib):
    """The Sec. III re-runs read each epoch's group steps from the library's
    schedule; the counts equal those of the oracle's draw (same geometry, seed)."""
    from paper_1709_00953_gb300 import experiments as X
    cfg = dict(geom=X.geometry_spec(),
               part=dict(tiles=(2, 2), view_blocks=X.N_VIEWS, det_blocks=(2, 1)))
    p, op = _pair(cfg)
    prm = dict(sampling=2, alpha=0.5, gamma=0.75, b=25.0, group_size=5, seed=X.SCHEDULE_SEED,
               theta_step=1.0 / 40.0)
    flat = lib.schedule_generate(p, prm, 3)
    rng = OS.SplitMix64(prm["seed"])
    P = OP.probability_table(op)
    vb = [op.row_block_parts(i)[0] for i in range(op.n_row_blocks)]
    eps = [OS.epoch_schedule(rng, P, prm, e, vb) for e in range(3)]
    assert flat == OS.flatten(eps)
    counts = X.groups_per_epoch(flat, 3)
    assert counts == [sum(len(g) for _, g in ep) for ep in eps]
    assert all(c > 0 for c in counts)


def test_explicit_view_sets_match_oracle(lib):
    """Row blocks over arbitrary view sets (Eq. e1 allows any index sets): an
    interleaved map view -> block gives the oracle's P table and schedule."""
    cfg = C.small_fan2d(n=64, views=30, nu=96, tiles=(2, 2), vb=3, du=2)
    vbo = [v % 3 for v in range(30)]
    g = lib.Geometry(cfg["geom"])
    p = lib.Partition(g, tiles=(2, 2), view_block_of=vbo, det_blocks=(2, 1))
    og = OGeom(**cfg["geom"])
    op = OPart(og, (2, 2), det_blocks=(2, 1), view_block_of=vbo)
    assert (p.m, p.n) == (op.n_row_blocks, op.n_col_blocks) == (6, 4)
    P = OP.probability_table(op)
    np.testing.assert_allclose(p.probabilities(), P, rtol=1e-12, atol=1e-15)
    prm = dict(cfg["solver"], sampling=2, alpha=0.5, group_size=2, seed=21)
    flat = lib.schedule_generate(p, prm, 3)
    rng = OS.SplitMix64(prm["seed"])
    vb = [op.row_block_parts(i)[0] for i in range(op.n_row_blocks)]
    eps = [OS.epoch_schedule(rng, P, prm, e, vb) for e in range(3)]
    assert flat == OS.flatten(eps)
