"""CPU emulation of the per-warp line-pair partition's control logic.

tests/csrc/emulate_stream.cpp runs the kernel's control decisions (PairCtl and
the stage map of csrc/lp_plan.h, the header the kernel uses) with plain copies
and asserts the hazards the GPU version must avoid: a line loaded twice or
written before it was taken, a stage refilled before it was taken or into the
wrong slot, a wrong mbarrier parity, and an unpartitioned or non-permuted
group.  Adversarial patterns (all / none / 1% / 99% predecessors,
alternating, sorted, reverse) are included.
"""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stream_control_emulation(tmp_path):
    exe = str(tmp_path / "emulate_stream")
    subprocess.run(["g++", "-O2", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2004_12532_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "csrc", "emulate_stream.cpp")],
                   check=True)
    for seed in (1, 2, 3):
        r = subprocess.run([exe, "1500", str(seed)], capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr


def test_plan_geometry_matches_oracle(orc):
    """The library's line map and X draw (lp_plan.h, compiled on the host)
    agree with the oracle's reading of Sec. 4 on sampled groups."""
    import ctypes
    src = r'''
#include "lp_plan.h"
extern "C" unsigned long long line_of(unsigned long long n, unsigned long long b,
    unsigned long long g, unsigned long long seed, unsigned long long level,
    unsigned long long i, unsigned long long j) {
  lp::StepGeom G = lp::make_geom(n, b, g, lp::level_seed(seed, level), 0);
  return lp::group_line(G, i, j);
}
'''
    import tempfile
    d = tempfile.mkdtemp()
    cpp = os.path.join(d, "g.cpp")
    so = os.path.join(d, "g.so")
    open(cpp, "w").write(src)
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    "-I", os.path.join(ROOT, "paper_2004_12532_gb300", "csrc"), "-o", so, cpp],
                   check=True)
    L = ctypes.CDLL(so)
    L.line_of.restype = ctypes.c_ulonglong
    L.line_of.argtypes = [ctypes.c_ulonglong] * 7
    n, b, g, seed, level = 1 << 16, 16, 37, 12345, 3
    s = orc.num_chunks(n, b, g)
    X = orc.draw_X(seed, level, s, g)
    for i in (0, 1, 17, 36):
        for j in range(s):
            assert L.line_of(n, b, g, seed, level, i, j) == j * g + (int(X[j]) + i) % g
