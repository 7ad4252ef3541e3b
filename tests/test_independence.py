"""The oracle and the CUDA path share no code: neither imports the other, the
CUDA sources include only their own headers and the public header, and the
benchmark reaches the oracle only from inside its CPU-baseline functions."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2605_17869_gb300")


def _py_files(d):
    for base, _, files in os.walk(d):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def _imported_modules(path, top_level_only=False):
    tree = ast.parse(open(path).read(), path)
    nodes = tree.body if top_level_only else ast.walk(tree)
    mods = set()
    for n in nodes:
        if isinstance(n, ast.Import):
            mods.update(a.name.split(".")[0] for a in n.names)
        elif isinstance(n, ast.ImportFrom) and n.level == 0 and n.module:
            mods.add(n.module.split(".")[0])
    return mods


def test_package_never_imports_the_oracle_or_the_input_generators():
    for f in _py_files(PKG):
        bad = _imported_modules(f) & {"oracle", "workloads"}
        assert not bad, (f, bad)


def test_oracle_never_imports_the_package():
    for f in _py_files(os.path.join(ROOT, "oracle")):
        assert "paper_2605_17869_gb300" not in _imported_modules(f), f


def test_cuda_sources_include_only_their_own_headers():
    csrc = os.path.join(PKG, "csrc")
    own = set(os.listdir(csrc))
    for f in sorted(os.listdir(csrc)):
        if not f.endswith((".cu", ".cuh", ".h", ".cpp")):
            continue
        for inc in re.findall(r'#include\s+"([^"]+)"', open(os.path.join(csrc, f)).read()):
            assert inc in own or inc == "../../include/sift_gb300.h", (f, inc)


def test_bench_imports_the_oracle_only_inside_functions():
    bench = os.path.join(ROOT, "bench.py")
    assert "oracle" not in _imported_modules(bench, top_level_only=True)
    tree = ast.parse(open(bench).read())
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for n in ast.walk(fn):
                if isinstance(n, ast.ImportFrom) and n.module and n.module.split(".")[0] == "oracle":
                    users.add(fn.name)
    assert users == {"_oracle_one"}, users
