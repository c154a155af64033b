"""Host logic of bench.py that needs no GPU."""
import os

import numpy as np
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _hash_of_copy(tmp_path, edit=None):
    import bench
    root = tmp_path / "r"
    for f in bench.KERNEL_SOURCES:
        dst = root / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copyfile(os.path.join(ROOT, f), dst)
    if edit:
        p = root / bench.KERNEL_SOURCES[0]
        p.write_text(edit(p.read_text()))
    old = bench.ROOT
    try:
        bench.ROOT = str(root)
        return bench.kernel_hash()
    finally:
        bench.ROOT = old


def test_kernel_hash_ignores_comments_but_not_code(tmp_path):
    """The stored ncu traffic figures are keyed by a hash of the kernel sources;
    editing a comment must keep the key, editing code must void it."""
    import bench
    base = _hash_of_copy(tmp_path)
    assert base == bench.kernel_hash()
    assert _hash_of_copy(tmp_path, lambda s: "// a new comment\n" + s.replace(
        "// ", "//  ", 3) + "\n/* trailing\n block */\n") == base
    assert _hash_of_copy(tmp_path, lambda s: s.replace("kConvThreads = 256", "kConvThreads = 128")) != base



def test_algorithmic_bytes_per_kernel():
    """4 bytes per FP32 value the method must move: r in and g out for the
    backprojection; x_J, g_J in and p, q out for the dual forward; p, q, z, r in
    and z, r out per ray, g_J per step and x_J, x^_J in and x^_J out per batch
    for the epilogue; x^ in, x and x^ out per voxel for the epoch close (and
    d, r in and r out per ray under epoch sync)."""
    import bench
    assert bench.algorithmic_bytes("backproject", 1000, 64) == 4 * (1000 + 64)
    assert bench.algorithmic_bytes("forward_dual", 1000, 64) == 4 * (2000 + 128)
    assert bench.algorithmic_bytes("epilogue", 10, 4) == 4 * (60 + 4 + 12)
    # 12 steps on one 64-voxel tile in one batch
    assert bench.algorithmic_bytes("epilogue", 100, 12 * 64, 64) == 4 * (600 + 768 + 192)
    assert bench.algorithmic_bytes("epoch_close", 10, 4) == 0
    assert bench.algorithmic_bytes("epoch_close", 0, 0, volume_voxels=1000) == 12000
    assert bench.algorithmic_bytes("epoch_close", 0, 0, volume_voxels=1000, epoch_rays=50) == 12600


def test_oracle_steps_split_groups_into_row_blocks():
    """The bounded CPU sample of a grouped workload takes the scheduled
    group's row blocks one at a time, in order, then the next group."""
    import bench
    from synth import configs as C
    cfg = C.small_cone3d(n=8, views=8, nd=12, tiles=(2, 1, 1), group=4, steps=4)
    y = np.random.default_rng(0).random(8 * 12 * 12).astype(np.float32)
    st = bench.OracleSteps(cfg, y)
    assert st.grouped
    j0, first = st.next()
    group = first + [i for _, (i,) in st.pending]
    assert len(group) == 4 and all(j == j0 for j, _ in st.pending)
    for i in group[1:]:
        assert st.next() == (j0, [i])
    assert len(st.next()[1]) == 1  # the next group starts
    dt, nz = st.step()
    assert dt >= 0 and nz >= 0 and len(st.o.log) == 1
