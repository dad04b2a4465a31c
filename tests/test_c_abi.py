"""The C ABI from plain C: tests/c/abi_check.c is compiled with gcc as C11 against
include/pic.h, linked to the built libpic.so and run; it checks the defaults and the argument
validation that answers before any device work (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_caller_compiles_links_and_validates(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2106_12919_gb300 import build
    libdir = os.path.dirname(build.LIB)
    if not os.path.exists(build.LIB):
        pytest.skip("libpic is not built")
    exe = str(tmp_path / "abi_check")
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c", "abi_check.c"), "-L", libdir, "-lpic", "-Wl,-rpath," + libdir,
           "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
