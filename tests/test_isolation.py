"""The oracle and the CUDA path share no code (CPU only, a scan of the sources).

* The package never imports the oracle, and the oracle never imports the package, except the
  seeded input generators (``inputs``), which hold none of the method's arithmetic.
* The oracle's modules import only numpy and the standard library.
* No C/CUDA source includes anything from the oracle's directory.
* ``bench.py`` reaches the oracle only in its CPU workers (the CPU baseline and the oracle's
  whole-pulse propagators for the precision table), and ``__graft_entry__.py`` only in
  ``smoke()``.
"""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1707_02162_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _py_files(d):
    for base, dirs, files in os.walk(d):
        dirs[:] = [x for x in dirs if x not in ("__pycache__", "_build", "build")]
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def _imports(path):
    """(module name, enclosing top-level function or None) of every import in a file."""
    tree = ast.parse(open(path).read(), filename=path)
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            f = fn
            if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) and fn is None:
                f = child.name
            if isinstance(child, ast.Import):
                out.extend((a.name, f) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = child.module or ""
                out.append((mod, f))
                if mod == "" or mod in ("oracle", "paper_1707_02162_gb300"):
                    out.extend((f"{mod}.{a.name}".lstrip("."), f) for a in child.names)
            visit(child, f)

    visit(tree, None)
    return out


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        for mod, _ in _imports(path):
            assert not mod.split(".")[0] == "oracle", f"{path} imports {mod}"


STDLIB_OK = {"__future__", "math", "fractions", "argparse", "os", "sys", "time", "numpy", "scipy",
             "scipy.optimize"}


def test_oracle_imports_only_numpy_stdlib_and_the_input_generators():
    for path in _py_files(ORACLE):
        for mod, _ in _imports(path):
            top = mod.split(".")[0]
            if top == "oracle":
                continue
            if top == "paper_1707_02162_gb300":
                assert mod in ("paper_1707_02162_gb300", "paper_1707_02162_gb300.inputs"), f"{path}: {mod}"
                assert os.path.basename(path) != "redo_oracle.py", "the oracle proper imports no package code"
                continue
            assert mod in STDLIB_OK, f"{path} imports {mod}"


def test_input_generators_import_neither_side():
    for mod, _ in _imports(os.path.join(PKG, "inputs.py")):
        assert mod.split(".")[0] in ("__future__", "dataclasses", "numpy"), mod


def test_no_native_source_includes_oracle_files():
    pat = re.compile(r'#\s*include\s*[<"]([^>"]+)[>"]')
    n = 0
    for base, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".cu", ".cuh", ".h", ".cpp", ".c")):
                n += 1
                for inc in pat.findall(open(os.path.join(base, f)).read()):
                    assert "oracle" not in inc, f"{f} includes {inc}"
    for f in os.listdir(os.path.join(ROOT, "include")):
        for inc in pat.findall(open(os.path.join(ROOT, "include", f)).read()):
            assert "oracle" not in inc
    assert n > 0


@pytest.mark.parametrize("fname,allowed", [("bench.py", {"_oracle_worker", "_oracle_parity_worker"}),
                                           ("__graft_entry__.py", {"smoke"})])
def test_oracle_reached_only_from_the_permitted_functions(fname, allowed):
    uses = [(m, f) for m, f in _imports(os.path.join(ROOT, fname)) if m.split(".")[0] == "oracle"]
    assert uses, f"{fname} is expected to use the oracle somewhere"
    for mod, fn in uses:
        assert fn in allowed, f"{fname}: {mod} imported in {fn!r}"
