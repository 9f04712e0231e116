"""The oracle and the CUDA library share no code: the package never imports the oracle, the
oracle never imports the package or includes its sources, the input generators (graphgen) import
neither, and bench.py reaches the oracle only from its CPU legs (run_reference, cpu_baseline) and,
to check the residuals of the scale-24 and scale-27 results after their timed solves, from the
legs that report them (config24, run_config)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1602_01421_gb300"


def _imports(path):
    """(top-level module name, enclosing function or None) of every import in a Python file."""
    tree = ast.parse(open(path).read())
    out = []

    def visit(node, func):
        for ch in ast.iter_child_nodes(node):
            f = ch.name if isinstance(ch, (ast.FunctionDef, ast.AsyncFunctionDef)) else func
            if isinstance(ch, ast.Import):
                out.extend((a.name.split(".")[0], func) for a in ch.names)
            elif isinstance(ch, ast.ImportFrom) and ch.level == 0 and ch.module:
                out.append((ch.module.split(".")[0], func))
            visit(ch, f)

    visit(tree, None)
    return out


def _py(dirname):
    return sorted(glob.glob(os.path.join(ROOT, dirname, "**", "*.py"), recursive=True))


def test_package_never_imports_the_oracle():
    files = _py(PKG)
    assert files
    for f in files:
        assert all(m != "oracle" for m, _ in _imports(f)), f


def test_oracle_never_imports_the_package():
    for f in _py("oracle"):
        assert all(m != PKG for m, _ in _imports(f)), f


def test_input_generators_import_neither():
    for f in _py("graphgen"):
        assert all(m not in ("oracle", PKG) for m, _ in _imports(f)), f


def test_native_sources_do_not_include_each_other():
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    for f in glob.glob(os.path.join(ROOT, PKG, "csrc", "*")):
        for h in inc.findall(open(f).read()):
            assert "oracle" not in h, (f, h)
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.c")) + glob.glob(os.path.join(ROOT, "oracle", "*.h")):
        for h in inc.findall(open(f).read()):
            assert "csrc" not in h and not h.startswith("fe") and "tc.cuh" not in h, (f, h)


def test_bench_uses_the_oracle_only_in_its_cpu_legs_and_result_checks():
    uses = [func for m, func in _imports(os.path.join(ROOT, "bench.py")) if m == "oracle"]
    assert uses and set(uses) <= {"run_reference", "cpu_baseline", "config24", "run_config"}, uses
    assert None not in uses                                 # never at module level
