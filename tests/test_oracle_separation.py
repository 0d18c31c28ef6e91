"""The oracle and the CUDA path share no code: a static check of the
sources.  The library package (the C-ABI sources and the Python binding)
neither imports, includes nor links anything under oracle/; the oracle
neither imports the package's binding nor includes its sources (both may
read the seeded input generators, paper_1603_02526_gb300/inputs.py, which
hold none of the method's arithmetic); and the benchmark and the entry
points touch the oracle only in their baseline, reference and checking
functions."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1603_02526_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _code(path):
    """Source text without comments and docstrings."""
    src = open(path).read()
    if path.endswith(".py"):
        t = ast.parse(src)
        for node in ast.walk(t):
            if isinstance(node, (ast.Module, ast.FunctionDef, ast.ClassDef, ast.AsyncFunctionDef)) and node.body:
                first = node.body[0]
                if isinstance(first, ast.Expr) and isinstance(getattr(first, "value", None), ast.Constant):
                    first.value.value = ""
        return ast.unparse(t)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"//[^\n]*", "", src)


def test_library_does_not_reach_the_oracle():
    bad = re.compile(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|fga_oracle|liboracle|\bog_[a-z_]+\s*\(|oracle/")
    for f in _files(PKG, (".py", ".cpp", ".cu", ".cuh", ".h")):
        hits = bad.findall(_code(f))
        assert not hits, (f, hits)
    for f in _files(os.path.join(ROOT, "include"), (".h",)):
        assert not bad.findall(_code(f)), f


def test_oracle_does_not_reach_the_library():
    bad = re.compile(r"paper_1603_02526_gb300\.(?!inputs\b)\w+|libfgadmm|fgadmm\.h|#include\s+\"(?:fga_|sweep|tile_|"
                     r"hinge_|mpc_|persist|residual|tc05)")
    for f in _files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")):
        hits = bad.findall(_code(f))
        assert not hits, (f, hits)


def test_bench_and_entry_touch_the_oracle_only_in_their_baselines():
    allowed = {"bench.py": {"oracle_sample", "cpu_baselines_other"},
               "__graft_entry__.py": {"build", "smoke"}}
    for name, funcs in allowed.items():
        t = ast.parse(open(os.path.join(ROOT, name)).read())
        for node in t.body:                                   # no module-level import of the oracle
            if isinstance(node, (ast.Import, ast.ImportFrom)):
                mods = [node.module] if isinstance(node, ast.ImportFrom) else [a.name for a in node.names]
                assert not any(m and m.split(".")[0] == "oracle" for m in mods), (name, mods)
        for node in ast.walk(t):
            if isinstance(node, ast.FunctionDef):
                for sub in ast.walk(node):
                    if isinstance(sub, (ast.Import, ast.ImportFrom)):
                        mods = [sub.module] if isinstance(sub, ast.ImportFrom) else [a.name for a in sub.names]
                        if any(m and m.split(".")[0] == "oracle" for m in mods):
                            assert node.name in funcs, (name, node.name)
