"""Host logic of the host-array partition (lp_partition_host_*), no GPU: the
chunk plan that decides the upload order and which device-to-host copies are
legal, compiled from the library's own header (csrc/lp_hostpart.h) and driven
with a serial partition in place of the device: it always finishes, leaves the
array partitioned with the right split and multiset, never writes a host
position before its chunk was read, and gives the same result however far
ahead the uploads run."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_chunk_plan(tmp_path):
    exe = str(tmp_path / "hostpart_test")
    subprocess.run(["g++", "-O2", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_2004_12532_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "csrc", "hostpart_test.cpp")],
                   check=True)
    r = subprocess.run([exe, "400"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "OK", r.stdout + r.stderr
