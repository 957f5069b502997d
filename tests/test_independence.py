"""The oracle and the CUDA path share no code.

Static checks over the sources: nothing in the product package (its Python
modules, the CUDA sources, the C header) imports, includes or loads anything
under oracle/, and the oracle imports nothing from the product package.  The
one module both sides may use is the seeded input generator
(paper_2105_11815_gb300/workloads.py), which holds none of the method's
arithmetic, and it imports neither side.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2105_11815_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            out.add(node.module.split(".")[0])
    return out


def _py_files(top):
    for d, _, files in os.walk(top):
        if "__pycache__" in d or "_lib" in d or "_build" in d:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(d, f)


def test_product_package_never_imports_the_oracle():
    for path in _py_files(PKG):
        assert "oracle" not in _imports(path), path


def test_cuda_sources_include_nothing_from_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h")):
            text = open(os.path.join(csrc, f)).read()
            for inc in re.findall(r'#include\s+"([^"]+)"', text):
                assert "oracle" not in inc, (f, inc)
    header = open(os.path.join(ROOT, "include", "skills.h")).read()
    assert "oracle" not in " ".join(re.findall(r'#include\s+"([^"]+)"', header))


def test_oracle_never_imports_the_product_package():
    for path in _py_files(ORACLE):
        assert "paper_2105_11815_gb300" not in _imports(path), path


def test_shared_generators_import_neither_side():
    imps = _imports(os.path.join(PKG, "workloads.py"))
    assert "oracle" not in imps
    # the generators load no CUDA library and none of the product's modules
    src = open(os.path.join(PKG, "workloads.py")).read()
    assert "ctypes" not in imps and "lib()" not in src
    assert not re.search(r"from \.\s*import|from \.(?!\.)\w", src)
