"""The C ABI from plain C: tests/c_client/client.c compiles against
include/gpchol.h alone (gcc, C11, no CUDA or C++ headers), links the built
libgpchol.so and runs the calls that need no device."""
import os
import shutil
import subprocess

import pytest

import paper_1907_01063_gb300 as gp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_client_compiles_links_and_runs(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = gp.library_path()
    libdir = os.path.dirname(lib)
    exe = tmp_path / "client"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_client", "client.c"), "-L", libdir, "-lgpchol",
                           f"-Wl,-rpath,{libdir}", "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FAIL" not in r.stdout
    assert r.stdout.count("ok ") == 13
