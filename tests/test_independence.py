"""The oracle and the CUDA path share no code, and the product path has no
CPU fallback (static checks; no GPU)."""
import ast
import glob
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2408_14558_gb300")

def imported_modules(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out

def test_oracle_does_not_import_the_package():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        assert "paper_2408_14558_gb300" not in imported_modules(f), f

def test_package_does_not_import_the_oracle():
    for f in glob.glob(os.path.join(PKG, "**", "*.py"), recursive=True):
        assert "oracle" not in imported_modules(f), f

def test_c_sources_include_nothing_of_the_other_side():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.c")) + glob.glob(os.path.join(ROOT, "oracle", "*.h")):
        inc = re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(f).read())
        assert not any(i.startswith("spg") or "spgemm1d" in i or i.endswith(".cuh") for i in inc), (f, inc)
    for f in glob.glob(os.path.join(PKG, "csrc", "*")):
        inc = re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(f).read())
        assert not any("oracle" in i for i in inc), (f, inc)

def test_missing_library_raises(tmp_path):
    """Without the built library every call fails loudly (a fresh interpreter,
    pointed at a path that does not exist)."""
    code = ("import paper_2408_14558_gb300 as g\n"
            "try:\n"
            f"    g.load_library({str(tmp_path / 'nope.so')!r})\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.stdout.startswith("raised"), out.stdout + out.stderr
