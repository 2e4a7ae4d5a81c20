"""The ctypes mirrors of the C-ABI structs in qpr.py have the layout that
include/qpr.h gives them: a small C program compiled against the header
prints every field's offset and every struct's size, and each must equal
the ctypes one (a field added to one side only would make the library read
the wrong option)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2003_04930_gb300 import qpr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [qpr.qpr_options, qpr.qpr_stats, qpr.qpr_profile, qpr.qpr_problem, qpr.qpr_gnn_sample,
           qpr.qpr_tune_result, qpr.qpr_rkf45_options, qpr.qpr_rkf45_stats]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "qpr.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'    printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


@pytest.mark.parametrize("st", STRUCTS, ids=lambda s: s.__name__)
def test_ctypes_struct_matches_header(c_layout, st):
    name = st.__name__
    assert ctypes.sizeof(st) == c_layout[(name, "sizeof")]
    for field, _ in st._fields_:
        assert getattr(st, field).offset == c_layout[(name, field)], field
