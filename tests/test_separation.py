"""The oracle and the GPU library stay independent of each other.

The oracle is test infrastructure: only the tests, the smoke check and the
benchmark's CPU legs may load it, and it shares no code, header or generated
table with the CUDA sources.  The seeded input generators are the one module
both sides are fed from, and they import neither.  These checks read the
sources (no build, no GPU)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1202_6163_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def files_under(d, exts):
    out = []
    for base, _, names in os.walk(d):
        if "__pycache__" in base:
            continue
        out += [os.path.join(base, n) for n in names if n.endswith(exts)]
    return sorted(out)


def imported_modules(path):
    """(top-level module, enclosing function or None) of every import in a Python file."""
    tree = ast.parse(open(path).read(), path)
    found = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                found.extend((a.name.split(".")[0], fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.level == 0 and child.module:
                found.append((child.module.split(".")[0], fn))
            visit(child, f)

    visit(tree, None)
    return found


NATIVE = (".cu", ".cuh", ".h", ".c", ".cpp")


def test_library_never_loads_or_includes_the_oracle():
    for path in files_under(PKG, (".py",)):
        mods = {m for m, _ in imported_modules(path)}
        assert "oracle" not in mods, path
        assert "liboracle" not in open(path).read(), path
    for path in files_under(PKG, NATIVE) + files_under(os.path.join(ROOT, "include"), NATIVE):
        src = open(path).read()
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', src):
            assert "oracle" not in inc, (path, inc)
        assert "pf_oracle" not in src and "liboracle" not in src, path


def test_oracle_uses_only_the_c_library():
    allowed = {"math.h", "stdint.h", "stdlib.h", "string.h", "stddef.h", "stdio.h", "float.h", "limits.h"}
    sources = files_under(ORACLE, NATIVE)
    assert sources, "the oracle's C source is missing"
    for path in sources:
        incs = re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read())
        assert set(incs) <= allowed, (path, set(incs) - allowed)
    for path in files_under(ORACLE, (".py",)):
        mods = {m for m, _ in imported_modules(path)}
        assert not mods & {"paper_1202_6163_gb300", "torch"}, (path, mods)


def test_input_generators_import_neither_side():
    mods = {m for m, _ in imported_modules(os.path.join(PKG, "workloads.py"))}
    assert mods <= {"__future__", "math", "numpy"}, mods


@pytest.mark.parametrize("name", ["bench.py", "__graft_entry__.py"])
def test_oracle_loaded_only_by_its_permitted_callers(name):
    # the benchmark loads the oracle only in its CPU-baseline and reference legs;
    # the entry module only in smoke() (build() compiles it, which is not using it)
    permitted = {"bench.py": {"oracle_step_time", "cpu_baseline", "cpu_baseline_batched", "run_reference"},
                 "__graft_entry__.py": {"smoke", "build"}}[name]
    for mod, fn in imported_modules(os.path.join(ROOT, name)):
        if mod == "oracle":
            assert fn in permitted, (name, fn)
