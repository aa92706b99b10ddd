"""The C-ABI library loads and exports every function include/unify.h declares,
and the Python mirror of unify_params_t has the C layout. No GPU work is done."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "unify.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"UNIFY_API\s+[\w\s\*]+?\b(unify_\w+)\s*\(", src)))


def _lib():
    import shutil
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    from paper_2412_02448_gb300 import buildlib as b
    return ctypes.CDLL(b.build())


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 9
    lib = _lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_params_layout_matches_header(tmp_path):
    import paper_2412_02448_gb300 as U
    prog = tmp_path / "p.c"
    prog.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "unify.h"\n'
                    'int main(void){unify_params_t p; printf("%zu %zu %zu %zu %zu\\n", sizeof p,'
                    ' offsetof(unify_params_t, tau_a), offsetof(unify_params_t, tau_b),'
                    ' offsetof(unify_params_t, cand_cap), offsetof(unify_params_t, scan_rows)); return 0;}\n')
    exe = tmp_path / "p"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    P = U.Params
    assert got == [ctypes.sizeof(P), P.tau_a.offset, P.tau_b.offset, P.cand_cap.offset, P.scan_rows.offset]
