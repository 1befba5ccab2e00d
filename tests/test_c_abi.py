"""The C ABI from C: tests/c/abi_host.c, compiled with gcc as C99 against
include/ilu.h and linked with libilu.so, runs its host-only checks (grid
helpers, host-only set-up, stencils, LFA, argument errors) without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_compiles_as_c_and_host_calls_work(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    import paper_2210_15280_gb300 as g
    g.build()
    so_dir = os.path.join(ROOT, "paper_2210_15280_gb300")
    exe = str(tmp_path / "abi_host")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_host.c"), "-o", exe, "-L", so_dir, "-lilu", "-lm",
           "-Wl,-rpath," + so_dir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FAIL" not in r.stdout
