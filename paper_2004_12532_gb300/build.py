"""Build libpartition.so in-tree with nvcc for sm_103a.

Each CUDA / C++ source in csrc/ is compiled to an object in parallel, then
linked into paper_2004_12532_gb300/libpartition.so.  Objects go to
paper_2004_12532_gb300/_build/ (git-ignored).  Rebuilds only what changed.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpartition.so")
YARD = os.path.join(PKG, "yardstick")
YLIB = os.path.join(PKG, "libyardstick.so")
CLIB = os.path.join(PKG, "libcpuyard.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpartition")
    return cand


def _deps():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _compile(src, extra):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    if not _stale(obj, [src] + _deps() + [__file__]):
        return obj
    cmd = [nvcc()] + ARCH + NVFLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    os.replace(obj + ".tmp", obj)
    return obj


def _link(target, objs, force):
    if force or _stale(target, objs):
        tmp = target + ".tmp%d" % os.getpid()
        # -ldl: the NVTX ranges look up a profiler's injection library at run time
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, target)


def build(verbose_ptxas: bool = False, force: bool = False) -> str:
    """Compile every source under csrc/ and link libpartition.so, and the
    out-of-place library yardstick (yardstick/) into libyardstick.so; return
    the path of libpartition.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force:
        for f in glob.glob(os.path.join(OUT_DIR, "*.o")):
            os.remove(f)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    ysrcs = sorted(glob.glob(os.path.join(YARD, "*.cu")))
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs) + len(ysrcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
        yobjs = list(ex.map(lambda s: _compile(s, extra), ysrcs))
    _link(LIB, objs, force)
    if yobjs:
        _link(YLIB, yobjs, force)
    _build_cpu_yardstick(force)
    return LIB


def _build_cpu_yardstick(force):
    """The host-core Smoothed Striding yardstick (yardstick/*.c, OpenMP)."""
    srcs = sorted(glob.glob(os.path.join(YARD, "*.c")))
    if not srcs or not (force or _stale(CLIB, srcs + [__file__])):
        return
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        return  # optional: the bench reports it as unavailable
    tmp = CLIB + ".tmp%d" % os.getpid()
    r = subprocess.run([cc, "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs,
                       capture_output=True, text=True)
    if r.returncode != 0:  # optional: the bench reports it as unavailable
        sys.stderr.write("note: host-core yardstick not built:\n%s\n" % r.stderr[-2000:])
        return
    os.replace(tmp, CLIB)


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv))
