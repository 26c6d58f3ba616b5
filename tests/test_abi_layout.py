"""The ctypes mirrors of include/pic.h's structs match the C layout (no GPU): a small C
program built here with gcc prints sizeof and the offset of every field the binding
declares, and the binding must agree byte for byte."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["pic_config", "pic_params", "pic_info", "pic_allocator", "pic_serve_config", "pic_result", "pic_peaks"]


@pytest.fixture(scope="module")
def P():
    from paper_2310_11393_gb300 import pic

    return pic


def c_layout(P):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pic.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(P, name)._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, key, val = line.split()
        got[(name, key)] = int(val)
    return got


def test_binding_structs_match_the_c_header(P):
    got = c_layout(P)
    for name in STRUCTS:
        st = getattr(P, name)
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)


def header_fields():
    """Field names of every typedef'd struct in include/pic.h, in declaration order."""
    import re

    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        names = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            fp = re.match(r".*\(\s*\*\s*(\w+)\s*\)\s*\(", decl)       # function pointer
            if fp:
                names.append(fp.group(1))
                continue
            parts = decl.split(",")
            first = re.sub(r"\[.*?\]", "", parts[0]).split()[-1].lstrip("*")
            names.append(first)
            names += [re.sub(r"\[.*?\]", "", p).strip().lstrip("*") for p in parts[1:]]
        out[name] = names
    return out


def test_binding_declares_every_header_field_in_order(P):
    hf = header_fields()
    for name in STRUCTS:
        assert [f for f, _ in getattr(P, name)._fields_] == hf[name], name
