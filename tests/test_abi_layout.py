"""CPU check that the Python binding's ctypes structures have exactly the layout of the C header's
structures: a small C program compiled with the host compiler against include/rte.h prints the
size of every structure and the offset of every field, and the test compares them with ctypes'
(a field added to the header but not to the binding, or in another order, would otherwise pass
garbage across the boundary without any error)."""
import os
import shutil
import subprocess

import pytest

from paper_2402_10488_gb300 import rte

HERE = os.path.dirname(os.path.abspath(__file__))
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

STRUCTS = {
    "rte_disc_desc": rte._DiscDesc,
    "rte_rom_opts": rte._RomOpts,
    "rte_solve_opts": rte._SolveOpts,
    "rte_solve_report": rte.SolveReport,
    "rte_gmres_opts": rte._GmresOpts,
    "rte_serve_report": rte.ServeReport,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rte.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", INCLUDE, str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def test_binding_structures_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert layout[(cname, "size")] == __import__("ctypes").sizeof(py), cname
        for fname, _ in py._fields_:
            assert layout[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def _header_fields():
    """Field names of each typedef'd structure in include/rte.h, in declaration order."""
    import re
    text = open(os.path.join(INCLUDE, "rte.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        names = []
        for decl in m.group(1).split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):          # "int nx, ny" declares two fields
                names.append(re.findall(r"(\w+)\s*(?:\[\w*\])?\s*$", part.strip())[0])
        out[m.group(2)] = names
    return out


def test_binding_declares_every_header_field_in_order():
    fields = _header_fields()
    for cname, py in STRUCTS.items():
        assert fields[cname] == [f for f, _ in py._fields_], cname
