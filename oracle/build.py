"""Compile the C oracle into oracle/liboracle.so with the host gcc.

The oracle is test infrastructure: only tests/, __graft_entry__.smoke() and
bench.py's CPU legs load it.  Plain C, portable flags (no -march=native), so
the same source builds on x86_64 and aarch64 hosts.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
HDR = os.path.join(HERE, "oracle.h")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Build liboracle.so if missing or older than its sources; return its path."""
    if not force and os.path.exists(LIB):
        lib_m = os.path.getmtime(LIB)
        if lib_m >= os.path.getmtime(SRC) and lib_m >= os.path.getmtime(HDR):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
