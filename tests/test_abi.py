"""The C-ABI library builds, loads and exports every symbol of include/lbdd.h.

CPU only: no call here reaches a kernel (argument checks and host-side
helpers only).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbdd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbdd_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2304_06543_gb300 as lb
    return lb.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_built_for_sm_103a():
    import paper_2304_06543_gb300._build as b
    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)
    assert os.path.exists(b.LIB)


def test_host_side_calls(lib):
    import paper_2304_06543_gb300 as lb
    assert lb.strerror(0) == "ok"
    assert "invariant" in lb.strerror(-5)
    assert lb.cm_pitch(500, lb.CM_I16) == 504
    assert lb.cm_pitch(501, lb.CM_I32) == 504
    assert lb.best_transfer_workspace(0, 5) == 0
    h = ctypes.c_void_p()
    # argument errors are reported before any CUDA call
    assert lib.lbdd_create(ctypes.byref(h), 0, 5, None, 0, 0, None, None, None) == lb.ERR_ARG
    assert h.value is None
    assert lib.lbdd_solve(None, -1) == lb.ERR_ARG
    lib.lbdd_destroy(None)


@pytest.mark.parametrize("n,k", [(1, 300), (3, 256), (20, 500), (200000, 500), (140000, 512),
                                 (2000000, 2000), (9000, 4096), (50, 7)])
def test_best_transfer_workspace_covers_every_path(lib, n, k):
    """The scan's workspace holds, at least, the allotted units grouped by
    center (4n), the packed k x k table (8k^2), the work items (16 (n/64 + k)),
    and for 256..512 centers the row-order path's per-range key tables: 32-bit
    keys in up to 32 ranges (int16) or 64-bit keys in up to 16 (int32), both
    4k^2 x min(32, n) bytes."""
    import paper_2304_06543_gb300 as lb
    need = 4 * n + 8 * k * k + 16 * (n // 64 + k)
    if 256 <= k <= 512:
        need += 4 * k * k * min(32, n)
    assert lb.best_transfer_workspace(n, k) >= need


def test_product_does_not_reference_oracle():
    """The CUDA path and its binding never import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_2304_06543_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src
                assert "asral_oracle" not in src and "_oracle.so" not in src


def test_header_is_plain_c_and_a_c_program_links(tmp_path):
    """include/lbdd.h is a C header (C11, pedantic, no warnings) and a C
    program links against the library and calls it without any Python."""
    import subprocess
    import paper_2304_06543_gb300._build as b
    src = tmp_path / "t.c"
    src.write_text(
        '#include <stdio.h>\n#include "lbdd.h"\n'
        "int main(void) {\n"
        "  lbdd_solver* s = 0;\n"
        "  int rc = lbdd_create(&s, 0, 5, 0, LBDD_CM_I32, 0, 0, 0, 0);\n"
        '  printf("%d %lld %d\\n", rc, (long long)lbdd_cm_pitch(500, LBDD_CM_I16),\n'
        "         (int)lbdd_max_centers());\n"
        "  return rc == LBDD_ERR_ARG && s == 0 ? 0 : 1;\n}\n")
    exe = tmp_path / "t"
    libdir = os.path.dirname(b.LIB)
    out = subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
                          "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir,
                          "-l:" + os.path.basename(b.LIB), f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                         capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, run.stdout + run.stderr
    rc, pitch, kmax = run.stdout.split()
    assert int(pitch) == 504 and int(kmax) > 0


def test_every_exported_c_symbol_is_declared():
    """No undocumented entry points: the library's exported lbdd_* C symbols
    are exactly the functions include/lbdd.h declares."""
    import shutil
    import subprocess
    import paper_2304_06543_gb300._build as b
    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    out = subprocess.run(["nm", "-D", "--defined-only", b.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines()
                       if ln.split() and ln.split()[-1].startswith("lbdd_")})
    assert exported == declared_functions()
