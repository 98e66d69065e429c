"""The binding's ctypes structures match the C ABI of include/pifepic.h field by
field: a small C program built against the header prints the size of every
struct and the offset of every field, and the ctypes layouts must agree.  No
GPU: the program only includes the header."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C type name -> binding class name and its fields (in the binding's order)
STRUCTS = {
    "pifepic_mesh_desc": "MeshDesc",
    "pifepic_solver_desc": "SolverDesc",
    "pifepic_object_desc": "ObjectDesc",
    "pifepic_face_bc": "FaceBC",
    "pifepic_stats": "Stats",
}


def _binding():
    from paper_2011_10214_gb300 import build
    if not os.path.exists(build.LIB):
        build.build_library()
    from paper_2011_10214_gb300 import capi
    return capi


def test_ctypes_layouts_match_the_header():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    capi = _binding()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pifepic.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        cls = getattr(capi, pyname)
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    import ctypes
    for cname, pyname in STRUCTS.items():
        cls = getattr(capi, pyname)
        assert ctypes.sizeof(cls) == got[(cname, "size")], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == got[(cname, fname)], (cname, fname)
