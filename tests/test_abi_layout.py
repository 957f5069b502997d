"""The ctypes structures of the Python binding have the C header's layout.

A small C program compiled against include/skills.h with the host compiler
prints sizeof and the offset of every field of ski_matrix, ski_opts and
ski_info; the binding's ctypes.Structure classes must agree field by field
(names, offsets, sizes) and in total size.  No GPU and no CUDA headers are
needed: the header is plain C.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2105_11815_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = (pkg.ski_matrix, pkg.ski_opts, pkg.ski_info)


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "skills.h"', "int main(void) {"]
    for S in STRUCTS:
        name = S.__name__
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in S._fields_:
            lines.append('  printf("%s %s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (name, field, name, field, name, field))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes, fields = {}, {}
    for line in out:
        parts = line.split()
        if len(parts) == 3 and parts[1] == "sizeof":
            sizes[parts[0]] = int(parts[2])
        elif len(parts) == 4:
            fields[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return sizes, fields


def test_ctypes_structures_match_the_header(tmp_path):
    sizes, fields = _c_layout(tmp_path)
    for S in STRUCTS:
        name = S.__name__
        assert ctypes.sizeof(S) == sizes[name], name
        for field, ctype in S._fields_:
            off, size = fields[(name, field)]
            assert getattr(S, field).offset == off, (name, field)
            assert ctypes.sizeof(ctype) == size, (name, field)
        # every member of the C struct appears in the binding: the fields'
        # sizes add up to the struct size less its trailing padding
        last = S._fields_[-1][0]
        assert getattr(S, last).offset + ctypes.sizeof(S._fields_[-1][1]) <= sizes[name]
