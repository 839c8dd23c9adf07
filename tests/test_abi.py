"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/libpartition.h declares.  No GPU needed."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:lp_status|uint64_t|uint32_t|const char \*|void)\s+\*?\s*"
                             r"(lp_[a-z0-9_]+)\s*\(", text):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2004_12532_gb300 import build
    return build.build()


def test_headers_declare_functions():
    names = declared_functions()
    assert "lp_partition_u64" in names and "lp_ctx_create" in names
    assert len(names) >= 15


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_functions() if getattr(lib, n, None) is None]
    assert not missing, missing


def test_binding_covers_declared_symbols():
    from paper_2004_12532_gb300 import binding
    missing = [n for n in declared_functions() if n not in binding._SIGS]
    assert not missing, missing


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_2004_12532_gb300 import binding
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError):
        binding.lib()


def test_builds_for_sm103a_only():
    # the one target architecture of every compile (no PTX for other targets)
    from paper_2004_12532_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_header_is_plain_c(tmp_path):
    """include/libpartition.h compiles as C99 and as C++17 (a C ABI: plain
    pointers and sizes, no C++ or torch types), and a C program can take the
    address of every entry point it declares."""
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    inc = os.path.join(root, "include")
    cuda_inc = "/usr/local/cuda/include"
    names = declared_functions()
    body = "\n".join("  (void)&%s;" % n for n in names)
    src = tmp_path / "use.c"
    src.write_text('#include "libpartition.h"\nint main(void) {\n%s\n  return 0;\n}\n' % body)
    for cc, std in (("gcc", "-std=c99"), ("g++", "-std=c++17")):
        if shutil.which(cc) is None:
            pytest.skip("no %s" % cc)
        args = [cc, std, "-Wall", "-Werror", "-fsyntax-only", "-I", inc, "-I", cuda_inc]
        if cc == "g++":
            args += ["-x", "c++"]
        r = subprocess.run(args + [str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
