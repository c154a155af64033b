"""Host logic of bench.py that needs no GPU."""
import os
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

