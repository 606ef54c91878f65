"""The oracle and the CUDA path stay independent, read from the sources (no GPU): the package
never imports the oracle or the tests, the oracle never imports the package, the C and CUDA
sources include nothing from outside the package and include/, and outside the tests the oracle
is reached only by bench.py's CPU baseline and reference arm and by the smoke check of
__graft_entry__.py."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2305_07026_b300")


def _py_files(d):
    for base, _, files in os.walk(d):
        if "__pycache__" in base:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def _imports(path):
    """(module name, enclosing function or None) of every import in a file."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                out.append(((child.module or ""), fn))
            visit(child, f)
    visit(tree, None)
    return out


def _top(name):
    return name.split(".")[0]


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod, _ in _imports(path):
            assert _top(mod) not in ("oracle", "tests"), (path, mod)


def test_oracle_never_imports_the_package():
    for path in _py_files(os.path.join(ROOT, "oracle")):
        for mod, _ in _imports(path):
            assert _top(mod) not in ("paper_2305_07026_b300", "tests", "bench"), (path, mod)


def test_oracle_reached_only_by_the_cpu_legs():
    allowed = {
        "bench.py": {"cpu_oracle", "_oracle_block_worker", "cpu_oracle_all_cores", "run_reference",
                     "run_reference_batch"},
        "__graft_entry__.py": {"smoke"},
    }
    for name, fns in allowed.items():
        found = [(mod, fn) for mod, fn in _imports(os.path.join(ROOT, name)) if _top(mod) == "oracle"]
        assert found, name   # the legs exist
        for mod, fn in found:
            assert fn in fns, (name, mod, fn)


def test_native_sources_include_only_their_own_headers():
    csrc = os.path.join(PKG, "csrc")
    dirs = (os.path.realpath(csrc), os.path.realpath(os.path.join(ROOT, "include")))
    for f in os.listdir(csrc):
        for inc in re.findall(r'#include\s+"([^"]+)"', open(os.path.join(csrc, f)).read()):
            path = os.path.realpath(os.path.join(csrc, inc))
            assert os.path.exists(path) and os.path.dirname(path) in dirs, (f, inc)


def test_binding_fails_loudly_without_the_library(tmp_path):
    """With no compiled library beside it, the binding raises ImportError at import, and so do
    the package's loader and the modules that import the binding at load time; the others import
    it when first used, and no context can be made without it: there is no CPU fallback."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2305_07026_b300"
    pkg.mkdir()
    for f in ("__init__.py", "_lib.py", "partition.py"):
        shutil.copy(os.path.join(PKG, f), pkg / f)
    for code in ("import paper_2305_07026_b300._lib", "import paper_2305_07026_b300.partition",
                 "import paper_2305_07026_b300 as p; p.load()"):
        run = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True,
                             env={**os.environ, "PYTHONPATH": str(tmp_path)}, timeout=120)
        assert run.returncode != 0 and "is not built" in run.stderr, (code, run.stderr[-500:])
