"""The oracle and the CUDA path stay independent (no GPU): neither imports the other, the
package's sources never name the oracle in code, and outside tests/ only smoke() and
the benchmark's CPU-baseline function import it."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2502_08034_gb300")


def _imports(path):
    """(module name, enclosing function or None) of every import in a Python file."""
    tree = ast.parse(open(path).read())
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import):
                out.extend((a.name, fn) for a in child.names)
            elif isinstance(child, ast.ImportFrom) and child.module:
                out.append((child.module, fn))
            visit(child, f)

    visit(tree, None)
    return out


def _py_files(folder):
    for dirpath, _, files in os.walk(folder):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def test_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        mods = [m for m, _ in _imports(path)]
        assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), path


def test_native_sources_do_not_refer_to_the_oracle():
    for name in os.listdir(os.path.join(PKG, "csrc")):
        src = open(os.path.join(PKG, "csrc", name)).read()
        code = re.sub(r"//[^\n]*|/\*.*?\*/", " ", src, flags=re.S)
        assert "oracle" not in code, name


def test_oracle_never_imports_the_package():
    for path in _py_files(os.path.join(ROOT, "oracle")):
        mods = [m for m, _ in _imports(path)]
        assert not any(m.startswith("paper_2502_08034_gb300") for m in mods), path


def test_only_smoke_and_the_cpu_baseline_import_the_oracle_outside_tests():
    # bench.py: the functions of its CPU-baseline leg (the oracle's rate on one core and
    # on every core, and its serial time to steady state)
    allowed = {"__graft_entry__.py": {"smoke"},
               "bench.py": {"oracle_sample", "_oracle_slab", "oracle_time_to_steady"}}
    for name, fns in allowed.items():
        users = {fn for m, fn in _imports(os.path.join(ROOT, name))
                 if m == "oracle" or m.startswith("oracle.")}
        assert users <= fns, (name, users)
