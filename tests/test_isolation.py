"""Isolation of the product path: the package never imports the oracle (nor the oracle the
package's compute), and the binding refuses to load without the CUDA library (no fallback)."""
import ast
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2106_12919_gb300")


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.add(node.module.split(".")[0])
    return out


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                assert "oracle" not in _imports(os.path.join(dirpath, f)), f
    for dirpath, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            src = open(os.path.join(dirpath, f), errors="ignore").read()
            assert "oracle/" not in src and "oracle." not in src, f


def test_oracle_never_imports_the_package_compute():
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith(".py"):
            assert "paper_2106_12919_gb300" not in _imports(os.path.join(ROOT, "oracle", f)), f


def test_binding_refuses_to_load_without_the_library(tmp_path):
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2106_12919_gb300 import build\n"
            "build.LIB = %r\n"
            "try:\n"
            "    from paper_2106_12919_gb300 import pic\n"
            "except ImportError as e:\n"
            "    print('refused:', e)\n"
            "else:\n"
            "    print('loaded')\n") % (ROOT, str(tmp_path / "missing" / "libpic.so"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("refused:"), r.stdout + r.stderr


def test_bench_uses_the_oracle_only_for_its_cpu_legs():
    """bench.py imports the oracle only inside run_oracle_sample (the cpu_baseline and the
    reference arm), never at module level or on the timed path."""
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    top = set()
    for node in tree.body:
        if isinstance(node, ast.Import):
            top.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            top.add(node.module.split(".")[0])
    assert "oracle" not in top
    users = [f.name for f in ast.walk(tree) if isinstance(f, ast.FunctionDef)
             and any(isinstance(n, ast.ImportFrom) and n.module and n.module.split(".")[0] == "oracle"
                     for n in ast.walk(f))]
    assert users == ["run_oracle_sample"], users
