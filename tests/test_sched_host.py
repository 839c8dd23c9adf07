"""Host logic of the serving engine, no GPU: the device-memory arena behind
the HBM budget (no overlap, alignment, exact accounting, coalescing back to
one free run) and the FIFO admission rule (slot limit, budget, no
overtaking), compiled from the library's own header (csrc/lp_sched.h)."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arena_and_admission(tmp_path):
    exe = str(tmp_path / "sched_test")
    subprocess.run(["g++", "-O2", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2004_12532_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "csrc", "sched_test.cpp")],
                   check=True)
    r = subprocess.run([exe, "20000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
