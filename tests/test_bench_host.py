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
    for f in bench.PART_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_hash()
    target = dst / bench.PART_SOURCES[0]
    text = target.read_text()
    target.write_text(text + "\n// a comment only\n\n")
    assert bench.kernel_hash() == h0
    target.write_text(text + "\nstatic int lp_hash_probe_ = 1;\n")
    assert bench.kernel_hash() != h0



def test_profiled_traffic_follows_the_hash(tmp_path, monkeypatch):
    """A summary feeds roofline.traffic, scaled by the launch's units, only
    while its hash matches the kernel sources; otherwise the reason is given."""
    src = os.path.join(bench.ROOT, "paper_2004_12532_gb300", "csrc")
    root = tmp_path / "r"
    dst = root / "paper_2004_12532_gb300" / "csrc"
    dst.mkdir(parents=True)
    (root / "profiles").mkdir()
    for f in bench.PART_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    fname = bench.PROFILES["partition_u64"][0]
    summary = root / "profiles" / fname
    summary.write_text("kernel_sources_sha256_16: %s\ndram_bytes_per_key: 15.5\n"
                       % bench.kernel_hash(bench.PART_SOURCES))
    assert bench.profiled_traffic("partition_u64", 1000) == (15500.0, None)
    v, why = bench.profiled_traffic("partition_u32", 1000)
    assert v is None and "dram_bytes_per_key_u32" in why
    summary.write_text("kernel_sources_sha256_16: 0000000000000000\ndram_bytes_per_key: 15.5\n")
    v, why = bench.profiled_traffic("partition_u64", 1000)
    assert v is None and "changed" in why
