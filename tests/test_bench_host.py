"""Host logic of bench.py, no GPU: the hash that decides whether the committed
ncu summary still describes the partition kernel (roofline.traffic) ignores
comments and blank lines but not code."""
import os
import shutil

import bench


def test_kernel_hash_ignores_comments_not_code(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2004_12532_gb300", "csrc")
    root = tmp_path / "r"
    dst = root / "paper_2004_12532_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_hash()
    target = dst / bench.KERNEL_SOURCES[0]
    text = target.read_text()
    target.write_text(text + "\n// a comment only\n\n")
    assert bench.kernel_hash() == h0
    target.write_text(text + "\nstatic int lp_hash_probe_ = 1;\n")
    assert bench.kernel_hash() != h0

