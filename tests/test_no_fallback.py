"""The product path has no CPU fallback (no GPU needed): nothing in the
package imports the oracle, the benchmark and the entry module import it
only in their CPU-baseline, reference-arm, build and smoke functions, and
without a CUDA device the binding raises instead of computing."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2304_00140_gb300")


def _oracle_imports(path):
    """(enclosing function or None, line) of every import of the oracle"""
    tree = ast.parse(open(path).read(), path)
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            names = []
            if isinstance(child, ast.Import):
                names = [a.name for a in child.names]
            elif isinstance(child, ast.ImportFrom):
                names = [child.module or ""]
            if any(n == "oracle" or n.startswith("oracle.") for n in names):
                found.append((func, child.lineno))
            visit(child, f)
    visit(tree, None)
    return found


def test_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                assert _oracle_imports(os.path.join(dirpath, f)) == [], f
    for dirpath, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            src = open(os.path.join(dirpath, f), errors="replace").read()
            assert "oracle.h" not in src and "or_stage" not in src, f


def test_benchmark_and_entry_import_the_oracle_only_where_allowed():
    allowed = {"bench.py": {"cpu_oracle_rate", "run_reference"}, "__graft_entry__.py": {"build", "smoke"}}
    for name, funcs in allowed.items():
        imports = _oracle_imports(os.path.join(ROOT, name))
        assert imports, name
        for func, line in imports:
            assert func in funcs, (name, func, line)


def test_binding_raises_without_a_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2304_00140_gb300 import fv, workloads as wl
    with pytest.raises(RuntimeError, match="CUDA device"):
        fv.Solver(wl.advection(n=8))
