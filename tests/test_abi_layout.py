"""The ctypes mirrors of the C ABI structs match the header: a C program
compiled against include/nm_dose.h prints sizeof and every field's offset,
and the Python binding's structures must agree field by field."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2111_11687_gb300 import nmdose

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["nm_grid", "nm_materials", "nm_options", "nm_counters", "nm_conv3d_desc", "nm_denoise_options"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nm_dose.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(nmdose, name)
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {(a, b): int(c) for a, b, c in (l.split() for l in out.splitlines())}


def test_ctypes_structs_match_header(tmp_path):
    c = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(nmdose, name)
        assert ctypes.sizeof(cls) == c[(name, "sizeof")], name
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == c[(name, f)], (name, f)
